// io_reduce.h -- moment import/export and FP64 reductions.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "storage.cuh"

namespace hlbm {

// src: public layout [nb][10][512] (rho, u, S) of dtype 0 = f64, 1 = f32 (device).
cudaError_t import_moments(int storage, const void* src, int dtype, void* dst, int64_t n_nodes, const Scales* sc,
                           cudaStream_t s);

// dst: public layout; physical != 0 subtracts F/(2 rho) from u (F per node or uniform fu).
cudaError_t export_moments(int storage, const void* src, void* dst, int dtype, int64_t n_nodes, const Scales* sc,
                           const float* F, const double* fu, int physical, cudaStream_t s);

// Adds the level's mass, momentum and kinetic energy (times vol) to out[0..4]
// (device).  part is scratch of reduce_scratch_doubles(nb) doubles.  Blocks
// with skip[b] != 0 are left out.
cudaError_t reduce_level(int storage, const void* src, int64_t nb, const Scales* sc, const uint8_t* skip,
                         const float* F, const double* fu, double vol, double* part, double* out, cudaStream_t s);
// CTAs of the reduction over nb blocks, and the scratch it needs.
int reduce_ctas(int64_t nb);
size_t reduce_scratch_doubles(int64_t nb);

// Adds to *count (device) a positive number if any of the n values of a
// device buffer of dtype 0 = f64, 1 = f32 is not finite (nothing otherwise).
cudaError_t count_nonfinite(const void* buf, int dtype, int64_t n, unsigned long long* count, cudaStream_t s);

// Scales (reduced-precision storages) from the amax of a public-layout buffer
// (dtype 0 = f64, 1 = f32, device).  amax: scratch of 10 unsigned.
cudaError_t scales_from_public(const void* src, int dtype, int64_t nb, Scales* sc, unsigned* amax, cudaStream_t s);
// Recompute the scales of a stored buffer from its amax and re-encode it in
// place (no-op for FP32 / FP64 storage).  tmp: a second Scales in device memory.
cudaError_t rescale_storage(int storage, void* buf, int64_t nb, Scales* cur, Scales* tmp, unsigned* amax,
                            cudaStream_t s);
// The same, re-encoding a second buffer that shares the scales (the other
// ping-pong buffer of a level) with the same change of scales.
cudaError_t rescale_storage_both(int storage, void* buf, void* other, int64_t nb, Scales* cur, Scales* tmp,
                                 unsigned* amax, cudaStream_t s);
// The same for a buffer holding blocks of n_dom domains with their own scales:
// dom[b] is block b's domain, cur / tmp hold n_dom Scales, amax n_dom * 10.
cudaError_t rescale_storage_domains(int storage, void* buf, int64_t nb, const int32_t* dom, int n_dom, Scales* cur,
                                    Scales* tmp, unsigned* amax, cudaStream_t s);

}  // namespace hlbm
