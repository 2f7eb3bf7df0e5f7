"""Fault paths that need no GPU fault: non-finite inputs are refused before
they reach the state, and a state that blows up is reported.

* hlbm_write_moments with a NaN (host buffer) or an infinity (device buffer)
  returns HLBM_E_NONFINITE and leaves the level as it was, in FP32 and
  FP16-scaled storage;
* hlbm_set_force with a non-finite force or fluid fraction returns
  HLBM_E_NONFINITE, and a finite call afterwards succeeds;
* an unstable run (tau close to 1/2, velocities near the lattice speed of
  sound) is reported as HLBM_E_NONFINITE by hlbm_reduce; the context stays
  usable (a new lattice steps normally afterwards).
"""
import numpy as np
import pytest
import torch

from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_nonfinite_moments_are_refused(storage):
    shape = (16, 16, 16)
    M = wl.random_field(shape, 51, du=0.02)
    with hl.Lattice((16, 16, 16), tau=0.7, storage=storage) as lat:
        lat.set_dense()
        lat.write_moments(hl.dense_to_blocks(M))
        before = lat.read_moments()
        bad = hl.dense_to_blocks(M)
        bad[3, 5, 17] = np.nan
        with pytest.raises(hl.HlbmError) as ei:
            lat.write_moments(bad)
        assert ei.value.code == hl.E_NONFINITE
        assert np.array_equal(lat.read_moments(), before)
        dev = torch.tensor(hl.dense_to_blocks(M).astype(np.float32), device="cuda")
        dev[1, 2, 3] = float("inf")
        with pytest.raises(hl.HlbmError) as ei:
            lat.write_moments(dev)
        assert ei.value.code == hl.E_NONFINITE
        assert np.array_equal(lat.read_moments(), before)


def test_nonfinite_force_fields_are_refused():
    with hl.Lattice((16, 16, 16), tau=0.7, storage="f32") as lat:
        lat.set_dense()
        F = torch.zeros((8, 3, 512), dtype=torch.float32, device="cuda")
        eps = torch.ones((8, 512), dtype=torch.float32, device="cuda")
        F[2, 1, 7] = float("nan")
        with pytest.raises(hl.HlbmError) as ei:
            lat.set_force(F, eps)
        assert ei.value.code == hl.E_NONFINITE
        F[2, 1, 7] = 0.0
        eps[4, 9] = float("-inf")
        with pytest.raises(hl.HlbmError) as ei:
            lat.set_force(F, eps)
        assert ei.value.code == hl.E_NONFINITE
        eps[4, 9] = 1.0
        lat.set_force(F, eps)
        lat.step(2)
        assert np.isfinite(lat.reduce()).all()


def test_blow_up_is_reported_and_the_context_survives():
    shape = (16, 16, 16)
    g = np.random.default_rng(52)
    ux = 0.9 * np.sign(g.standard_normal(shape))
    M = wl.equilibrium_field(np.ones(shape), ux, -ux, 0.5 * ux)
    with hl.Lattice((16, 16, 16), tau=0.5005, storage="f32") as lat:
        lat.set_dense()
        lat.write_moments(hl.dense_to_blocks(M))
        code = None
        for _ in range(40):
            lat.step(25)
            try:
                lat.reduce()
            except hl.HlbmError as e:
                code = e.code
                break
        assert code == hl.E_NONFINITE
    with hl.Lattice((16, 16, 16), tau=0.7, storage="f32") as lat:
        lat.set_dense()
        lat.write_moments(hl.dense_to_blocks(wl.random_field(shape, 53, du=0.02)))
        lat.step(4)
        assert np.isfinite(lat.reduce()).all()
