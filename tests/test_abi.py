"""The C ABI library builds, loads and exports every symbol include/homelbm.h declares.

CPU only: no compute call is made (there is no GPU here); calls that fail
before touching the device are checked for their error codes.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_14982_gb300 import build as B
from paper_2603_14982_gb300 import homelbm as hl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hl.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "homelbm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hlbm_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("hlbm_create", "hlbm_set_dense", "hlbm_set_force", "hlbm_step", "hlbm_read_moments",
                 "hlbm_write_moments", "hlbm_reduce", "hlbm_destroy", "hlbm_get_blocks", "hlbm_set_blocks"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(hl.exported_symbols()) <= set(declared_symbols())


def test_version_and_null_handling(lib):
    assert b"sm_103a" in lib.hlbm_version()
    assert lib.hlbm_destroy(None) == hl.OK
    assert lib.hlbm_step(None, 1) == hl.E_INVALID_ARG
    assert lib.hlbm_set_dense(None) == hl.E_INVALID_ARG


@pytest.mark.parametrize("kw,code", [
    (dict(extent=(20, 16, 16)), hl.E_INVALID_ARG),          # not a multiple of 8
    (dict(extent=(16, 16, 16), tau=0.5), hl.E_INVALID_ARG),  # tau must exceed 1/2
    (dict(extent=(16, 16, 16), storage=9), hl.E_INVALID_ARG),
    # post-collision rescale factor k_up = -249 between the two levels (|k| > 100 outside FP64)
    (dict(extent=(16, 128, 16), levels=2, tau=1.002, storage="f32"), hl.E_INVALID_ARG),
])
def test_create_rejects_bad_config(lib, kw, code):
    with pytest.raises(hl.HlbmError) as ei:
        hl.Lattice(**kw)
    assert ei.value.code == code


def test_config_struct_layout_matches_c():
    # int32 x5, pad, double, int32 x3, int32 x3, pad, void*, int32, pad
    assert ctypes.sizeof(hl.Config) == 72
    assert hl.Config.tau_finest.offset == 24
    assert hl.Config.stream.offset == 56


def test_layout_marshalling_roundtrip():
    g = np.random.default_rng(0)
    M = g.standard_normal((10, 16, 24, 8))
    Mb = hl.dense_to_blocks(M)
    assert Mb.shape == (2 * 3 * 1, 10, 512)
    # node (x, y, z) = (3, 9, 12) is block (0, 1, 1), cell 3 + 8*1 + 64*4
    assert Mb[0 + 1 * 1 + 1 * 3, 4, 3 + 8 + 256] == M[4, 12, 9, 3]
    assert np.array_equal(hl.blocks_to_dense(Mb, (16, 24, 8)), M)


@pytest.mark.parametrize("domains,storage", [
    ([], "f16s"),                                  # no domain
    ([((16, 16, 16), 0.6), ((20, 16, 16), 0.6)], "f16s"),   # not a multiple of 8
    ([((16, 16, 16), 0.5)], "f32"),                # tau must exceed 1/2
])
def test_batch_create_rejects_bad_domains(lib, domains, storage):
    with pytest.raises(hl.HlbmError) as ei:
        hl.Batch(domains, storage=storage)
    assert ei.value.code == hl.E_INVALID_ARG


def test_batch_rejects_fp64_and_non_periodic_domains(lib):
    with pytest.raises(hl.HlbmError) as ei:
        hl.Batch([((16, 16, 16), 0.6)], storage="f64")
    assert ei.value.code == hl.E_UNSUPPORTED
    cfg = (hl.Config * 1)()
    cfg[0].nx = cfg[0].ny = cfg[0].nz = 16
    cfg[0].block_edge, cfg[0].num_levels, cfg[0].tau_finest = 8, 1, 0.6
    cfg[0].periodic[0], cfg[0].periodic[1], cfg[0].periodic[2] = 1, 0, 1
    cfg[0].storage = hl.STORE_F32
    h = ctypes.c_void_p()
    assert lib.hlbm_batch_create(cfg, 1, ctypes.byref(h)) == hl.E_INVALID_ARG
    assert not h.value
    assert b"periodic" in lib.hlbm_batch_last_error(None)
    assert lib.hlbm_batch_destroy(None) == hl.OK
    assert lib.hlbm_batch_step(None, 1) == hl.E_INVALID_ARG


def test_binding_refuses_buffers_that_are_not_float32():
    """Buffers the library reads as float32 (force, fluid fraction, particle
    positions, adjoints) are refused in another dtype instead of being
    reinterpreted; a CPU tensor is refused where a device pointer is needed."""
    import torch
    from paper_2603_14982_gb300 import homelbm as hl
    with pytest.raises(TypeError):
        hl._f32(np.zeros((4, 3)), "positions")
    with pytest.raises(TypeError):
        hl._f32(torch.zeros(4, dtype=torch.float64), "eps")
    with pytest.raises(TypeError):
        hl._f32(torch.zeros(4, dtype=torch.float32), "eps", device=True)
    p, dev = hl._f32(np.zeros((4, 3), np.float32), "positions")
    assert dev == 0 and p.value is not None
