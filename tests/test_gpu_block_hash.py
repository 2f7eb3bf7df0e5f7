"""The spatial-hash block table (hlbm_set_block_lookup mode 1) against the
dense slot tables: everything that finds a block by position (neighbour
tables, interface transfers, the moment carry-over of a rebuild, the particle
deposit, the multi-level adjoint, open-face neighbour tables) must give the
same results bit for bit.

* a three-level falling cloud with rebuilds, deposits, drag and steps, the
  mode switched both ways between rebuilds;
* the two-level adjoint;
* open faces set after the blocks (neighbour tables rebuilt through the hash);
* bad modes and an injected allocation failure during the conversion.
"""
import numpy as np
import pytest
import torch

from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl
from tests.helpers import ml_adjoint_case

pytestmark = pytest.mark.gpu

EXT, L, PER = (128, 128, 128), 3, (True, False, True)


def state(lat, levels):
    return [lat.read_moments(level=l, dtype=np.float32) for l in range(levels)]


def blocks(lat, levels):
    return [lat.blocks(l)[0] for l in range(levels)] + [lat.interface_nodes(l, w) for l in range(levels)
                                                        for w in (0, 1)]


def run_cloud(switches):
    """Rebuild / deposit / step on the falling cloud; switches[k] is the block
    lookup mode set before rebuild k (None: leave it)."""
    pos0 = wl.particle_cloud(EXT[0], count=20000, seed=9, box=(0.25, 0.4, 0.25), y0_frac=0.2)
    out = []
    with hl.Lattice(EXT, levels=L, tau=0.9, periodic=PER, storage="f32") as lat:
        for k, t in enumerate(range(0, 48, 12)):
            if switches[k] is not None:
                lat.set_block_lookup(switches[k])
            pos = wl.fall(pos0, t)
            lat.rebuild_from_particles(pos)
            mode, nbytes = lat.block_lookup()
            slots = [(EXT[0] >> (3 + l)) * (EXT[1] >> (3 + l)) * (EXT[2] >> (3 + l)) for l in range(L)]
            stored = [lat.num_blocks(l) for l in range(L)]
            if mode == 0:
                assert nbytes == 4 * sum(slots)
            else:  # a hash of 2 to 4 entries of 12 bytes per block; empty levels keep their slot table
                lo = sum(24 * n if n else 4 * s for n, s in zip(stored, slots))
                hi = sum(12 * max(64, 4 * n) if n else 4 * s for n, s in zip(stored, slots))
                assert lo <= nbytes <= hi
            if k == 0:
                for l in range(L):
                    n = lat.num_blocks(l)
                    M = np.zeros((n, 10, 512))
                    M[:, 0] = 1.0
                    M[:, 1] = 0.02
                    M[:, 4] = 0.02 ** 2
                    lat.write_moments(M, level=l)
            lat.deposit_particles(pos)
            lat.set_drag(1e-3, (0.0, -0.01, 0.0), 2)
            lat.step(8)
            out.append((blocks(lat, L), state(lat, L)))
    return out


def assert_same(a, b):
    for (ba, sa), (bb, sb) in zip(a, b):
        for x, y in zip(ba, bb):
            assert np.array_equal(x, y)
        for x, y in zip(sa, sb):
            assert np.array_equal(x, y)


def test_hash_lookup_matches_slot_tables_over_rebuilds():
    dense = run_cloud([None, None, None, None])
    hashed = run_cloud([1, None, None, None])
    assert_same(dense, hashed)
    switched = run_cloud([None, 1, 0, 1])  # converted in place between rebuilds
    assert_same(dense, switched)


def test_hash_lookup_adjoint_matches():
    c = ml_adjoint_case("two_level")
    z, y, x = np.nonzero(c["O0"])
    per = 1 << (c["L"] - 1)
    grads = []
    for mode in (0, 1):
        with hl.Lattice(c["ext"], levels=c["L"], tau=c["tau0"], periodic=c["periodic"], storage="f32") as lat:
            lat.set_block_lookup(mode)
            lat.set_fine_blocks(np.stack([x, y, z], axis=1))
            coords = [lat.blocks(l)[0] for l in range(c["L"])]
            for l in range(c["L"]):
                lat.write_moments(hl.dense_to_blocks(c["M0"][l], coords[l]), level=l)
            F = torch.tensor(hl.dense_to_blocks(c["F"].astype(np.float32), coords[0]), device="cuda")
            lat.set_force(F)
            lat.forward_record(c["n_coarse"] * per, c["ckpt"] * per)
            W = torch.cat([torch.tensor(hl.dense_to_blocks(c["W"][l].astype(np.float32), coords[l]), device="cuda")
                           for l in range(c["L"])])
            grads.append(lat.adjoint(W, torch.empty_like(F)).cpu().numpy())
    assert np.array_equal(grads[0], grads[1])
    assert np.abs(grads[0]).max() > 0


def test_hash_lookup_with_open_faces():
    ext = (16, 128, 16)
    O0 = np.zeros((2, 16, 2), bool)
    O0[:, 7:9, :] = True
    z, y, x = np.nonzero(O0)
    res = []
    for mode in (0, 1):
        with hl.Lattice(ext, levels=2, tau=0.8, periodic=(False, True, True), storage="f32") as lat:
            lat.set_block_lookup(mode)
            lat.set_fine_blocks(np.stack([x, y, z], axis=1))
            lat.set_open_faces([hl.FACE_INLET, hl.FACE_OUTFLOW, 0, 0, 0, 0], 0.04, 0.3, 1.5, 1)
            lat.step(4)
            res.append(state(lat, 2))
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_block_lookup_arguments_and_failed_conversion():
    with hl.Lattice(EXT, levels=L, tau=0.9, periodic=PER, storage="f32") as lat:
        with pytest.raises(hl.HlbmError) as ei:
            lat.set_block_lookup(2)
        assert ei.value.code == hl.E_INVALID_ARG
        pos = wl.particle_cloud(EXT[0], count=5000, seed=3, box=(0.25, 0.4, 0.25), y0_frac=0.2)
        lat.rebuild_from_particles(pos)
        lat.step(4)
        before = state(lat, L)
        try:
            hl.inject_alloc_failure(1)  # the first table goes through, the second fails
            with pytest.raises(hl.HlbmError) as ei:
                lat.set_block_lookup(1)
            assert ei.value.code == hl.E_OOM
        finally:
            hl.inject_alloc_failure(-1)
        lat.deposit_particles(pos)  # the slot tables are still in place
        lat.set_block_lookup(1)
        lat.step(4)
        after_hash = state(lat, L)
    with hl.Lattice(EXT, levels=L, tau=0.9, periodic=PER, storage="f32") as ref:
        ref.rebuild_from_particles(pos)
        ref.step(4)
        assert all(np.array_equal(a, b) for a, b in zip(state(ref, L), before))
        ref.deposit_particles(pos)
        ref.step(4)
        assert all(np.array_equal(a, b) for a, b in zip(state(ref, L), after_hash))
