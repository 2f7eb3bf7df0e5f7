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
// (device).  part is scratch of nb*7 doubles.  Blocks with skip[b] != 0 are left out.
cudaError_t reduce_level(int storage, const void* src, int64_t nb, const Scales* sc, const uint8_t* skip,
                         const float* F, const double* fu, double vol, double* part, double* out, cudaStream_t s);

}  // namespace hlbm
