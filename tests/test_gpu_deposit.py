"""Particle deposit (hlbm_deposit_particles) against the oracle's deposit.

The GPU fields must equal oracle.deposit.fields (FP64 rounded once to
float32) exactly.  There is no getter for the fields, so each case steps the
lattice once with the deposited fields and once with the oracle's fields
passed through hlbm_set_force: the two results must be bit-identical.
"""
import numpy as np
import pytest
import torch

from oracle import deposit as dp
from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def set_fields(lat, F, eps):
    lat.set_force(torch.tensor(F, dtype=torch.float32, device="cuda"),
                  torch.tensor(eps, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("moving", [True, False])
def test_single_level_deposit_matches_oracle(moving):
    ext = (32, 24, 16)
    shape = (16, 24, 32)
    g = np.random.default_rng(11)
    pos = (g.uniform(0, 1, (4000, 3)) * np.array(ext)).astype(np.float32)
    pos[:7] = np.array([-3.0, 5.0, 40.0], dtype=np.float32)    # clamped into the domain
    pos[7:10, 1] = np.nan                                       # dropped
    pos[10:500] = np.array([5.5, 6.5, 7.5], dtype=np.float32)   # eta saturates at 0.4
    M0b = hl.dense_to_blocks(wl.random_field(shape, 12, du=0.02))
    ok = np.isfinite(pos).all(axis=1)
    F, eps = dp.fields(pos[ok], shape, moving=moving)
    with hl.Lattice(ext, tau=0.9, periodic=(True, False, True)) as lat:
        lat.set_dense()
        lat.write_moments(M0b)
        dropped = lat.deposit_particles(pos, moving=moving)
        lat.step(1)
        got = lat.read_moments()
        lat.write_moments(M0b)
        set_fields(lat, hl.dense_to_blocks(F), hl.dense_to_blocks(eps[None])[:, 0])
        lat.step(1)
        ref = lat.read_moments()
    assert dropped == 3
    assert np.array_equal(got, ref)


def test_three_level_deposit_on_rebuilt_hierarchy():
    ext = (128, 128, 128)
    pos = wl.particle_cloud(128, count=60000, seed=13)
    with hl.Lattice(ext, levels=3, tau=0.9, periodic=(True, False, True)) as lat:
        lat.rebuild_from_particles(torch.tensor(pos, device="cuda"))
        coords, _ = lat.blocks(0)
        n = [lat.num_blocks(l) for l in range(3)]
        M0b = [None] * 3
        for l in range(3):
            e = 128 >> l
            M0b[l] = hl.dense_to_blocks(wl.random_field((e, e, e), 20 + l, du=0.01), lat.blocks(l)[0])
        def run(**kw):
            for l in range(3):
                lat.write_moments(M0b[l], level=l)
            if "pos" in kw:
                dropped = lat.deposit_particles(kw["pos"])
            else:
                set_fields(lat, *kw["fields"])
                dropped = None
            lat.step(4)
            return [lat.read_moments(level=l) for l in range(3)], dropped
        got, dropped = run(pos=torch.tensor(pos, device="cuda"))
        F, eps = dp.fields(pos, (128, 128, 128))
        ref, _ = run(fields=(hl.dense_to_blocks(F, coords), hl.dense_to_blocks(eps[None], coords)[:, 0]))
    assert dropped == 0   # every particle sits in a stored finest-level block
    assert n[0] > 0
    for l in range(3):
        assert np.array_equal(got[l], ref[l]), l
