"""Pins for the coupled step of the oracle (streaming only, drag exchange,
collision; Fig. 4 and Sec. 5.4).

* a uniform periodic flow relaxes to the sediment velocity by the closed form
  u'_n = v_p - (1 - k kappa eta)^(n/k) (v_p - u'_0) (exchange every k steps,
  rho = 1): the streamed velocity of a uniform field is its stored velocity,
  and each step adds F / rho to the stored velocity;
* with kappa = 0 the coupled step is the plain step with zero force;
* mass is conserved on a random field with solids;
* the multi-level driver with the drag reduces to ``run_coupled`` when the
  hierarchy has a single level.
"""
import numpy as np
import pytest
import torch

from oracle import coupling as cp
from oracle import hierarchy as hy
from oracle import multilevel as ml
from oracle import single_level as sl
from paper_2603_14982_gb300 import workloads as wl



@pytest.fixture(autouse=True)
def _fp64_default_dtype():
    """FP64 default dtype for the oracle's tensors, restored afterwards: the
    GPU tests collected in the same session must keep torch's float32 default."""
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    yield
    torch.set_default_dtype(old)


def uniform(shape, u):
    ux, uy, uz = (np.full(shape, v) for v in u)
    return torch.tensor(wl.equilibrium_field(np.ones(shape), ux, uy, uz))


def test_uniform_flow_relaxes_to_sediment_velocity():
    shape = (8, 8, 8)
    u0, vp, kappa, eta = (0.02, -0.01, 0.005), (0.01, 0.03, -0.02), 0.05, 0.3
    eps = torch.full(shape, 1.0 - eta)
    for every in (1, 2, 3):
        n = 4 * every
        M, _ = cp.run_coupled(uniform(shape, u0), n, 1.0, eps, vp, kappa, every)
        for a in range(3):
            want = vp[a] - (1.0 - every * kappa * eta) ** (n // every) * (vp[a] - u0[a])
            assert abs(M[1 + a].mean().item() - want) < 1e-15
            assert (M[1 + a] - M[1 + a].mean()).abs().max() < 1e-15
        assert (M[0] - 1.0).abs().max() < 1e-14


def test_zero_drag_is_the_plain_step():
    shape = (8, 16, 8)
    M0 = torch.tensor(wl.random_field(shape, 3, du=0.03))
    eps = torch.tensor(np.random.default_rng(4).uniform(0.6, 1.0, shape))
    Mc, F = cp.coupled_step(M0, 0.8, eps, (0.1, 0.0, 0.0), 0.0, periodic=(True, False, True))
    Mp = sl.step(M0, 0.8, force=None, eps=eps, periodic=(True, False, True))
    assert torch.equal(Mc, Mp)
    assert F.abs().max() == 0.0


def test_mass_conserved_with_drag_and_solids():
    shape = (16, 16, 16)
    M0 = torch.tensor(wl.random_field(shape, 7, du=0.03))
    solid = torch.zeros(shape, dtype=torch.bool)
    solid[5:9, 5:9, 5:9] = True
    eps = torch.tensor(np.random.default_rng(8).uniform(0.6, 1.0, shape))
    M, F = cp.run_coupled(M0, 6, 1.0, eps, (0.0, -0.05, 0.0), 0.1, 2, periodic=(True, True, True), solid=solid)
    assert abs(M[0].sum().item() - M0[0].sum().item()) < 1e-11 * M0[0].sum().item()
    assert F[:, solid].abs().max() == 0.0
    assert F.abs().max() > 0.0


def test_multilevel_driver_with_one_level_matches_run_coupled():
    ext = (16, 16, 16)
    h = hy.Hierarchy(np.zeros(hy.block_dims(ext, 8, 0), bool), ext, 8, 1, (True, True, True))
    M0 = torch.tensor(wl.random_field((16, 16, 16), 9, du=0.02))
    eps = torch.tensor(np.random.default_rng(10).uniform(0.7, 1.0, (16, 16, 16)))
    m = ml.MultiLevel(h, 0.75, eps=eps, drag=(0.05, (0.0, 0.02, 0.01), 3))
    m.set_level(0, M0)
    for _ in range(7):
        m.coarse_step()
    M, F = cp.run_coupled(M0, 7, 0.75, eps, (0.0, 0.02, 0.01), 0.05, 3)
    assert torch.equal(m.current(0), M)
    assert torch.equal(m.force, F)
