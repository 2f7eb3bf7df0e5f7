"""Pins for the oracle's reverse-mode gradient (dL/dF of the outlet kinetic energy).

The reverse-mode gradient is checked against the complex-step derivative
(exact to rounding for this forward model) and against central finite
differences, on a small channel with an obstacle; checkpointed and plain
reverse passes must agree.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as adj
from paper_2603_14982_gb300 import workloads as wl



@pytest.fixture(autouse=True)
def _fp64_default_dtype():
    """FP64 default dtype for the oracle's tensors, restored afterwards: the
    GPU tests collected in the same session must keep torch's float32 default."""
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    yield
    torch.set_default_dtype(old)


def setup(n=16, steps=10):
    shape = (n // 2, n // 2, n)
    solid = np.zeros(shape, dtype=bool)
    solid[2:6, 2:6, 6:10] = True
    M0 = wl.random_field(shape, 81, du=0.02, drho=1e-3, dneq=1e-4)
    M0[:, solid] = wl.rest_field((1, 1, 1))[:, 0, 0, :1]
    F = wl.noisy_force(shape, seed=82, mean=(1e-5, 0, 0), sigma=1e-5)
    return torch.tensor(M0), torch.tensor(F), torch.tensor(solid), steps


def test_reverse_mode_matches_complex_step():
    M0, F, solid, steps = setup()
    per = (True, False, False)
    L, g = adj.gradient(M0, F, steps, 0.7, per, solid=solid)
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = torch.tensor(rng.standard_normal(tuple(F.shape)))
        cs = adj.complex_step(M0, F, steps, 0.7, per, d, solid=solid)
        assert abs((g * d).sum().item() - cs) <= 1e-10 * abs(cs) + 1e-18


def test_reverse_mode_matches_central_differences():
    M0, F, solid, steps = setup()
    per = (True, False, False)
    _, g = adj.gradient(M0, F, steps, 0.7, per, solid=solid)
    rng = np.random.default_rng(4)
    for _ in range(2):
        d = torch.tensor(rng.standard_normal(tuple(F.shape)))
        h = 1e-5
        lp = adj.outlet_kinetic_energy(adj.run_forward(M0, F + h * d, steps, 0.7, per, solid), F + h * d)
        lm = adj.outlet_kinetic_energy(adj.run_forward(M0, F - h * d, steps, 0.7, per, solid), F - h * d)
        fd = ((lp - lm) / (2 * h)).item()
        assert abs((g * d).sum().item() - fd) <= 1e-5 * abs(fd)   # rounding-limited at h = 1e-5


def test_checkpointed_gradient_is_exact():
    M0, F, solid, steps = setup()
    per = (True, False, False)
    _, g1 = adj.gradient(M0, F, steps, 0.7, per, solid=solid)
    _, g2 = adj.gradient(M0, F, steps, 0.7, per, solid=solid, ckpt_every=3)
    assert torch.equal(g1, g2) or (g1 - g2).abs().max() < 1e-20


# ---------------------------------------------------------------- multi-level

def test_ml_finite_fill_leaves_stored_nodes_unchanged():
    """The multi-level derivatives give unstored nodes a finite rest state
    instead of NaN; stored nodes never read them, so the run is unchanged."""
    from oracle import multilevel as ml
    from tests.helpers import ml_adjoint_case
    c = ml_adjoint_case("two_level")
    Ms, _ = adj.ml_forward(c["h"], c["tau0"], c["M0"], torch.tensor(c["F"]), c["n_coarse"])
    m = ml.MultiLevel(c["h"], c["tau0"], force=torch.tensor(c["F"]))
    for l in range(c["L"]):
        m.set_level(l, c["M0"][l])
    for _ in range(c["n_coarse"]):
        m.coarse_step()
    for l in range(c["L"]):
        st = c["stored"][l]
        assert torch.equal(Ms[l][:, st], m.current(l)[:, st])
        assert torch.isfinite(Ms[l]).all()


def test_ml_reverse_mode_matches_complex_step():
    """dL/dF through sub-cycling, both transfers and their rescaling, on two
    and three levels (walls included): <g, d> equals the complex-step
    derivative along random directions and single cells."""
    from tests.helpers import ml_adjoint_case
    rng = np.random.default_rng(5)
    for name in ("two_level", "three_level_wall"):
        c = ml_adjoint_case(name)
        args = (c["h"], c["tau0"], c["M0"], c["F"], c["n_coarse"], c["W"])
        _, g = adj.ml_gradient(*args)
        assert g.abs().max() > 0
        dirs = [rng.standard_normal(c["F"].shape)]
        e = np.zeros(c["F"].shape)
        st0 = np.argwhere(c["stored"][0])
        z, y, x = st0[rng.integers(len(st0))]
        e[0, z, y, x] = 1.0
        dirs.append(e)
        for d in dirs:
            cs = adj.ml_complex_step(*args, d)
            assert abs((g.numpy() * d).sum() - cs) <= 1e-10 * abs(cs) + 1e-14, name
        # nodes level 0 does not store carry no gradient
        unstored = ~torch.as_tensor(c["stored"][0])
        if unstored.any():
            assert g[:, unstored].abs().max().item() == 0.0
