"""The coupled level-0 step (streaming only, drag exchange, collision; Fig. 4)
on the GPU against the oracle.

* single level with walls, a solid block and a random fluid fraction, drag
  exchanged every other step: FP32 within 1e-5 per step of the row scale,
  FP16-scaled storage within its per-step bound;
* two levels (a refined band), drag every other fine step: every level
  against the oracle's Algorithm 1 with the same coupled level-0 steps;
* a uniform flow relaxes to the sediment velocity by the closed form;
* argument checks, FP64 storage and the adjoint are refused while the drag is on.
"""
import numpy as np
import pytest
import torch

from oracle import coupling as cp
from oracle import hierarchy as hy
from oracle import multilevel as ml
from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl
from tests.helpers import rel_err, row_scales

pytestmark = pytest.mark.gpu

RP_TOL = {"f32": 1e-5, "f16s": 8 * 2.0 ** -11}
KAPPA, VP = 0.05, (0.01, -0.04, 0.02)


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_single_level_coupled_steps_match_oracle(storage):
    ext = (32, 16, 24)
    shape = (24, 16, 32)
    per = (True, False, True)
    solid = np.zeros(shape, dtype=bool)
    solid[8:14, 4:10, 10:18] = True
    M0 = wl.random_field(shape, 31, du=0.03)
    eps = np.random.default_rng(32).uniform(0.6, 1.0, shape).astype(np.float32)
    steps = 6
    with hl.Lattice(ext, tau=1.0, periodic=per, storage=storage) as lat:
        lat.set_dense()
        lat.set_solid(solid.astype(np.uint8))
        lat.write_moments(hl.dense_to_blocks(M0))
        start = hl.blocks_to_dense(lat.read_moments(), shape)
        lat.set_force(torch.zeros((lat.num_blocks(0), 3, 512), dtype=torch.float32, device="cuda"),
                      torch.tensor(hl.dense_to_blocks(eps[None]), device="cuda")[:, 0].contiguous())
        lat.set_drag(KAPPA, VP, 2)
        lat.step(steps)
        got = hl.blocks_to_dense(lat.read_moments(), shape)
    ref, F = cp.run_coupled(torch.tensor(start), steps, 1.0, torch.tensor(eps.astype(np.float64)), VP, KAPPA, 2,
                            periodic=per, solid=torch.tensor(solid))
    ref = ref.numpy()
    assert float(F.abs().max()) > 1e-4          # the drag is not negligible
    err = rel_err(got, ref, row_scales(ref, 0.03), mask=~solid)
    assert err.max() < steps * RP_TOL[storage], err


def test_two_level_coupled_steps_match_oracle():
    ext = (16, 128, 16)
    L = 2
    O0 = np.zeros(hy.block_dims(ext, 8, 0), bool)
    O0[:, 7:9, :] = True
    h = hy.Hierarchy(O0, ext, 8, L, (True, True, True))
    m0 = ml.MultiLevel(h, 0.8)
    lat = hl.Lattice(ext, levels=L, tau=0.8, periodic=(True, True, True), storage="f32")
    with lat:
        z, y, x = np.nonzero(O0)
        lat.set_fine_blocks(np.stack([x, y, z], axis=1))
        coords = [lat.blocks(l)[0] for l in range(L)]
        for l in range(L):
            X, Y, Z = m0.node_positions(l)
            ux = 0.01 * np.sin(2 * np.pi * Y / 128)
            M = wl.equilibrium_field(np.ones_like(ux) + 1e-3 * np.cos(2 * np.pi * X / 16), ux, 0.3 * ux,
                                     np.zeros_like(ux))
            lat.write_moments(hl.dense_to_blocks(M, coords[l]), level=l)
        start = [hl.blocks_to_dense(lat.read_moments(level=l), m0.shape[l], coords[l]) for l in range(L)]
        eps = np.random.default_rng(5).uniform(0.7, 1.0, m0.shape[0]).astype(np.float32)
        lat.set_force(torch.zeros((len(coords[0]), 3, 512), dtype=torch.float32, device="cuda"),
                      torch.tensor(hl.dense_to_blocks(eps[None], coords[0]), device="cuda")[:, 0].contiguous())
        lat.set_drag(KAPPA, VP, 2)
        m = ml.MultiLevel(h, 0.8, eps=torch.tensor(eps.astype(np.float64)), drag=(KAPPA, VP, 2))
        for l in range(L):
            m.set_level(l, start[l])
        for k in range(3):
            m.coarse_step()
            lat.step(2)
            for l in range(L):
                got = hl.blocks_to_dense(lat.read_moments(level=l), m.shape[l], coords[l])
                ref = m.current(l).numpy()
                err = rel_err(got, ref, row_scales(ref, 0.01), mask=m.stored[l].numpy())
                assert err.max() < 2e-5 * (k + 1), (k, l, err)


def test_uniform_flow_relaxes_on_the_gpu():
    u0, eta = (0.02, -0.01, 0.005), 0.3
    shape = (16, 16, 16)
    ux, uy, uz = (np.full(shape, v) for v in u0)
    M0 = wl.equilibrium_field(np.ones(shape), ux, uy, uz)
    with hl.Lattice((16, 16, 16), tau=1.0, storage="f32") as lat:
        lat.set_dense()
        lat.write_moments(hl.dense_to_blocks(M0))
        lat.set_force(torch.zeros((8, 3, 512), dtype=torch.float32, device="cuda"),
                      torch.full((8, 512), 1.0 - eta, dtype=torch.float32, device="cuda"))
        lat.set_drag(KAPPA, VP, 1)
        lat.step(8)
        got = lat.read_moments()
    e = np.float32(1.0) - np.float32(1.0 - eta)
    for a in range(3):
        want = VP[a] - (1.0 - KAPPA * float(e)) ** 8 * (VP[a] - u0[a])
        assert np.abs(got[:, 1 + a] - want).max() < 1e-6


def test_drag_arguments_and_refusals():
    with hl.Lattice((16, 16, 16), tau=0.7, storage="f32") as lat:
        lat.set_dense()
        with pytest.raises(hl.HlbmError) as ei:
            lat.set_drag(float("nan"), VP, 2)
        assert ei.value.code == hl.E_INVALID_ARG
        with pytest.raises(hl.HlbmError) as ei:
            lat.set_drag(KAPPA, VP, -1)
        assert ei.value.code == hl.E_INVALID_ARG
        lat.set_drag(KAPPA, VP, 2)
        with pytest.raises(hl.HlbmError) as ei:
            lat.forward_record(4, 2)
        assert ei.value.code == hl.E_UNSUPPORTED
        lat.set_drag(KAPPA, VP, 0)
        lat.forward_record(4, 2)
    with hl.Lattice((16, 16, 16), tau=0.7, storage="f64") as lat:
        lat.set_dense()
        with pytest.raises(hl.HlbmError) as ei:
            lat.set_drag(KAPPA, VP, 2)
        assert ei.value.code == hl.E_UNSUPPORTED
