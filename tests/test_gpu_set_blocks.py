"""Explicit hierarchies through hlbm_set_blocks (Sec. 5.1, 5.3, 6.1).

* an oracle hierarchy installed level by level gives the same block lists,
  flags and interface nodes as the oracle (and as the particle rebuild);
* a second explicit hierarchy carries the moments over like the oracle's
  rebuild, and its flags are the set differences against the first;
* a hierarchy that refines a region to level 1 only (a level-selection
  function with an intermediate level) runs Algorithm 1 to FP64 parity;
* every invariant has a refusal case, and a refused hierarchy leaves the
  lattice as it was.
"""
import numpy as np
import pytest

from oracle import hierarchy as hy
from oracle import multilevel as ml
from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl
from tests.test_gpu_multilevel import _compare, oracle_nodes, shear

pytestmark = pytest.mark.gpu

EXT, L, PER = (128, 128, 128), 3, (True, False, True)


def install(lat, h):
    for l in range(h.L):
        lat.set_blocks(l, h.blocks(l))


def assert_matches(lat, h, prev=None):
    for l in range(h.L):
        coords, flags = lat.blocks(l)
        assert np.array_equal(coords, h.blocks(l)), l
        assert np.array_equal(flags, h.flags(l, prev)), l
        for which in (0, 1):
            got = np.sort(lat.interface_nodes(l, which).astype(np.int64))
            assert np.array_equal(got, oracle_nodes(h, l, which)), (l, which)


def cloud_hierarchy(t=0):
    pos = wl.fall(wl.particle_cloud(128, count=20000, seed=9, box=(0.25, 0.4, 0.25), y0_frac=0.2), t)
    return pos, hy.from_particles(pos, EXT, 8, L, PER)


def test_explicit_hierarchy_equals_oracle_and_rebuild():
    pos, h = cloud_hierarchy()
    with hl.Lattice(EXT, levels=L, tau=0.9, periodic=PER) as lat, \
            hl.Lattice(EXT, levels=L, tau=0.9, periodic=PER) as ref:
        # levels staged in any order; the last one installs
        for l in (2, 0, 1):
            assert lat.num_blocks(0) == 0
            lat.set_blocks(l, h.blocks(l)[::-1])
        assert_matches(lat, h)
        ref.rebuild_from_particles(pos)
        for l in range(L):
            for which in (0, 1):
                assert np.array_equal(np.sort(lat.interface_nodes(l, which)), np.sort(ref.interface_nodes(l, which)))
        # a second hierarchy: flags against the first
        _, h2 = cloud_hierarchy(24)
        install(lat, h2)
        assert_matches(lat, h2, h)


def test_explicit_rebuild_moves_moments_like_the_oracle():
    ext, per = (32, 128, 32), (True, True, True)
    O0 = np.zeros(hy.block_dims(ext, 8, 0), bool)
    O0[1, 5:7, 1] = True
    h = hy.Hierarchy(O0, ext, 8, 2, per)
    m = ml.MultiLevel(h, 0.8)
    for l in range(2):
        X, Y, Z = m.node_positions(l)
        m.set_level(l, shear(0.01, 128)(X, Y, Z))
    with hl.Lattice(ext, levels=2, tau=0.8, periodic=per, storage="f64") as lat:
        install(lat, h)
        for l in range(2):
            coords, _ = lat.blocks(l)
            lat.write_moments(hl.dense_to_blocks(m.current(l).numpy(), coords), level=l)
        m.coarse_step()
        lat.step(2)
        O1 = np.zeros_like(O0)
        O1[1, 7:9, 2] = True
        h1 = hy.Hierarchy(O1, ext, 8, 2, per)
        m.rebuild(h1)
        install(lat, h1)
        assert_matches(lat, h1, h)
        _compare(lat, m, 1e-11, 0.01)
        m.coarse_step()
        lat.step(2)
        _compare(lat, m, 1e-11, 0.01)


def intermediate_hierarchy():
    """Three levels over 256 x 64 x 64: one occupied level-0 block, plus a
    region around level-2 block x = 5 refined to level 1 only."""
    ext = (256, 64, 64)
    O0 = np.zeros(hy.block_dims(ext, 8, 0), bool)
    O0[3, 3, 3] = True
    base = hy.Hierarchy(O0, ext, 8, L, PER)
    far = np.zeros_like(base.H[2])
    far[:, :, 5] = True
    H2 = base.H[2] | hy.dilate(far, PER)
    return ext, hy.Hierarchy.from_H([base.H[0], base.H[1], H2], ext, 8, L, PER), base


def test_intermediate_level_region_runs_algorithm1():
    ext, h, base = intermediate_hierarchy()
    assert (h.stored[1] & ~base.stored[1]).any() and all(len(h.blocks(l)) for l in range(L))
    m = ml.MultiLevel(h, 0.9)
    for l in range(L):
        X, Y, Z = m.node_positions(l)
        m.set_level(l, shear(0.005, 64)(X, Y, Z))
    with hl.Lattice(ext, levels=L, tau=0.9, periodic=PER, storage="f64") as lat:
        install(lat, h)
        assert_matches(lat, h)
        for l in range(L):
            coords, _ = lat.blocks(l)
            lat.write_moments(hl.dense_to_blocks(m.current(l).numpy(), coords), level=l)
        for _ in range(2):
            m.coarse_step()
            lat.step(4)
        _compare(lat, m, 1e-11, 0.005)


def _refused(lat, lists, words):
    with pytest.raises(hl.HlbmError) as e:
        for l, c in enumerate(lists):
            lat.set_blocks(l, c)
    assert e.value.code == hl.E_INVALID_ARG
    assert words in str(e.value), str(e.value)


def test_refusals_one_per_invariant():
    ext, _, h = intermediate_hierarchy()
    assert all(len(h.blocks(l)) for l in range(L)) and h.I[1].any()
    S = [h.blocks(l) for l in range(L)]
    with hl.Lattice(ext, levels=L, tau=0.9, periodic=PER) as lat:
        install(lat, h)
        before = [lat.blocks(l) for l in range(L)]
        # coordinates outside the grid (refused when staged)
        with pytest.raises(hl.HlbmError) as e:
            lat.set_blocks(0, np.array([[32, 0, 0]]))
        assert "outside" in str(e.value)
        # a block listed twice
        _refused(lat, [np.concatenate([S[0], S[0][:1]]), S[1], S[2]], "listed twice")
        # a stored internal block
        z, y, x = np.nonzero(h.I[1])
        _refused(lat, [S[0], np.concatenate([S[1], [[x[0], y[0], z[0]]]]), S[2]], "internal")
        # a stored block whose parent is neither stored nor internal
        z, y, x = np.nonzero(h.stored[1] & h.H[1] & ~h.I[1])
        keep = ~((S[1][:, 0] == x[0]) & (S[1][:, 1] == y[0]) & (S[1][:, 2] == z[0]))
        _refused(lat, [S[0], S[1][keep], S[2]], "neither stored nor internal")
        # a missing child of a refined block
        _refused(lat, [S[0][1:], S[1], S[2]], "all 8 must be stored")
        # the top level must cover every block that is not internal: drop a
        # level-2 block that has no children
        z, y, x = np.nonzero(h.stored[2] & ~h.H[2])
        keep = ~((S[2][:, 0] == x[0]) & (S[2][:, 1] == y[0]) & (S[2][:, 2] == z[0]))
        _refused(lat, [S[0], S[1], S[2][keep]], "top level")
        # no overlap: one level-1 block refined (not a union of 3x3x3 cubes)
        H1 = np.zeros_like(h.H[1])
        H1[1, 1, 4] = True
        bad = hy.Hierarchy.from_H([h.H[0], H1, hy.dilate(hy.parent(H1), PER)], ext, 8, L, PER)
        _refused(lat, [bad.blocks(l) for l in range(L)], "3x3x3")
        # 2:1 grading: level 2 not dilated around the level-1 region
        bad = hy.Hierarchy.from_H([h.H[0], h.H[1], hy.parent(h.H[1])], ext, 8, L, PER)
        _refused(lat, [bad.blocks(l) for l in range(L)], "2:1 grading")
        # every refusal left the installed hierarchy alone
        for l in range(L):
            got = lat.blocks(l)
            assert np.array_equal(got[0], before[l][0]) and np.array_equal(got[1], before[l][1])
