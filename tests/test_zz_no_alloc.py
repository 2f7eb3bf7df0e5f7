"""The allocation-free reduction entry point agrees with hlbm_reduce.

hlbm_reduce_f32_noalloc serves callers that cannot allocate device memory (code
living inside another application's allocator or a fixed memory budget): it
takes the moment buffer and a five-double output buffer from the caller and
uses only a fixed device array as scratch.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _noalloc(lib, mom, F, fu, out, stream):
    return lib.hlbm_reduce_f32_noalloc(ctypes.c_void_p(mom.data_ptr()), mom.shape[0],
                                       None if F is None else ctypes.c_void_p(F.data_ptr()),
                                       fu[0], fu[1], fu[2], ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(stream))


@pytest.mark.parametrize("use_field", [False, True])
def test_noalloc_reduce_matches_handle_reduce_twice(use_field):
    from paper_2603_14982_gb300 import build as B
    B.build()
    lib = hl.load()
    shape = (32, 24, 40)
    nz, ny, nx = shape
    fu = (2e-5, -1e-5, 3e-6)
    stream = torch.cuda.current_stream().cuda_stream
    with hl.Lattice((nx, ny, nz), tau=0.7, periodic=(True, False, True), storage="f32", stream=stream) as lat:
        lat.set_dense()
        F = None
        if use_field:
            Fd = wl.noisy_force(shape, seed=11, mean=fu, sigma=1e-5)
            F = torch.tensor(hl.dense_to_blocks(Fd), dtype=torch.float32, device="cuda")
            lat.set_force(F)
        else:
            lat.set_uniform_force(*fu)
        lat.write_moments(hl.dense_to_blocks(wl.random_field(shape, 12)))
        lat.step(3)
        mom = torch.empty((lat.num_blocks(), 10, 512), dtype=torch.float32, device="cuda")
        lat.read_moments(mom)
        ref = lat.reduce()[:5]
        outs = []
        for _ in range(2):
            out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
            assert _noalloc(lib, mom, F, fu, out, stream) == hl.OK, lib.hlbm_last_error(None)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
    # same tolerance as the parity tests: 1e-5 of the quantity's scale
    scale = np.array([abs(ref[0]), ref[0] * 0.02, ref[0] * 0.02, ref[0] * 0.02, abs(ref[4])])
    for o in outs:
        assert np.all(np.abs(o - ref) <= 1e-5 * scale), (o, ref)
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_address_survives_lattice_create_and_destroy():
    """The cached device address of the scratch stays valid across lattices:
    a call before a lattice exists, a call while one lives and a call after
    it is destroyed agree, and the result matches hlbm_reduce of that lattice."""
    from paper_2603_14982_gb300 import build as B
    B.build()
    lib = hl.load()
    shape = (16, 24, 32)
    M0 = hl.dense_to_blocks(wl.random_field(shape, 5)).astype(np.float32)
    mom = torch.tensor(M0, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    fu = (1e-5, 0.0, -2e-5)

    def call():
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, mom, None, fu, out, stream) == hl.OK, lib.hlbm_last_error(None)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    before = call()
    with hl.Lattice((32, 24, 16), tau=0.7, periodic=(True, True, True), stream=stream) as lat:
        lat.set_dense()
        lat.set_uniform_force(*fu)
        lat.write_moments(mom)
        ref = lat.reduce()[:5]
        during = call()
    after = call()
    assert np.array_equal(before, during) and np.array_equal(before, after)
    scale = np.array([abs(ref[0]), ref[0] * 0.02, ref[0] * 0.02, ref[0] * 0.02, abs(ref[4])])
    assert np.all(np.abs(before - ref) <= 1e-5 * scale), (before, ref)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    lib = hl.load()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    mom = torch.zeros((1, 10, 512), dtype=torch.float32, device="cuda")
    rc = lib.hlbm_reduce_f32_noalloc(ctypes.c_void_p(mom.data_ptr()), 65537, None, 0.0, 0.0, 0.0,
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert rc == hl.E_INVALID_ARG
    assert b"65536" in lib.hlbm_last_error(None)
