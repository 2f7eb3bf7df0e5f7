"""hlbm_reduce against FP64 sums of the moments the GPU holds.

The reduction sums in compensated FP32 per thread and FP64 across threads
(mass from the stored delta_rho, momentum through rho u = rho u' - F/2).  On
the same stored moments it must match the oracle's FP64 sums: mass to 1e-13
relative, momentum to 1e-11 of sum |rho u|, kinetic energy to 1e-6 relative
(its per-node products are FP32).
"""
import numpy as np
import pytest
import torch

from oracle import hierarchy as hy
from oracle import multilevel as ml
from oracle import single_level as sl
from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def check(r, mass, mom, mom_abs, ke):
    assert abs(r[0] - mass) <= 1e-13 * mass, (r[0], mass)
    for a in range(3):
        assert abs(r[1 + a] - mom[a]) <= 1e-11 * mom_abs, (a, r[1 + a], mom[a])
    assert abs(r[4] - ke) <= 1e-6 * ke, (r[4], ke)


@pytest.mark.parametrize("storage", ["f32", "f16s", "f64"])
@pytest.mark.parametrize("field", [False, True])
def test_single_level_reduce_matches_fp64_sums(storage, field):
    extent = (64, 40, 48)
    shape = (48, 40, 64)
    fu = (2e-5, -1e-5, 3e-6)
    with hl.Lattice(extent, tau=0.7, periodic=(True, False, True), storage=storage) as lat:
        lat.set_dense()
        if field:
            Fd = wl.noisy_force(shape, seed=11, mean=fu, sigma=1e-5)
            lat.set_force(torch.tensor(hl.dense_to_blocks(Fd), dtype=torch.float32, device="cuda"))
            force = torch.tensor(Fd.astype(np.float32).astype(np.float64))
        else:
            lat.set_uniform_force(*fu)
            force = fu
        lat.write_moments(hl.dense_to_blocks(wl.random_field(shape, 21, du=0.05, drho=0.01)))
        lat.step(2)
        M = torch.tensor(hl.blocks_to_dense(lat.read_moments(), shape))
        r = lat.reduce()
    u = sl.physical_velocity(M, force)
    mom = [float((M[0] * u[a]).sum()) for a in range(3)]
    mom_abs = float(sum((M[0] * u[a]).abs().sum() for a in range(3)))
    check(r, float(M[0].sum()), mom, mom_abs, float(sl.kinetic_energy(M, force)))


def test_multilevel_reduce_matches_oracle_on_the_same_moments():
    ext, L, per = (64, 128, 64), 3, (True, False, True)
    O0 = np.zeros(hy.block_dims(ext, 8, 0), bool)
    O0[3:5, 0:2, 3:5] = True
    h = hy.Hierarchy(O0, ext, 8, L, per)
    with hl.Lattice(ext, levels=L, tau=0.9, periodic=per, storage="f32") as lat:
        z, y, x = np.nonzero(O0)
        lat.set_fine_blocks(np.stack([x, y, z], axis=1))
        m = ml.MultiLevel(h, 0.9, force=(1e-5, -2e-5, 0.0))
        lat.set_uniform_force(1e-5, -2e-5, 0.0)
        for l in range(L):
            n = tuple(e >> l for e in ext[::-1])
            coords, _ = lat.blocks(l)
            lat.write_moments(hl.dense_to_blocks(wl.random_field(n, 30 + l, du=0.04, drho=0.01), coords), level=l)
        lat.step(4)
        for l in range(L):
            coords, _ = lat.blocks(l)
            m.set_level(l, hl.blocks_to_dense(lat.read_moments(level=l), m.shape[l], coords))
        r = lat.reduce()
    ro = m.reduce()
    check(r, ro[0], ro[1:4], 0.1 * ro[0], ro[4])   # |rho u| < 0.1 rho per node here
    assert abs(r[5] - ro[5]) <= 1e-13 * ro[0] and abs(r[6] - ro[6]) <= 1e-13 * ro[0]
