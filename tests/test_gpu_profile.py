"""The per-handle profile (hlbm_set_profiling / hlbm_get_profile): spans are
counted per kernel class, times are positive, profiling off records
nothing, reset zeroes the totals, and the results of a run do not depend on
whether it was profiled."""
import numpy as np
import pytest

from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_single_level_profile_counts():
    with hl.Lattice((32, 32, 32), tau=0.6, periodic=(True, False, False), storage="f32") as lat:
        lat.set_dense()
        lat.step(3)
        assert all(c == 0 for _, c in lat.profile().values())  # off by default
        lat.set_profiling(True)
        lat.step(10)
        lat.reduce()
        p = lat.profile()
        assert p["stream_collide"][1] == 10 and p["stream_collide"][0] > 0
        assert p["reduce"][1] == 1
        lat.set_profiling(False)
        lat.step(5)
        assert lat.profile(reset=True)["stream_collide"][1] == 10
        assert lat.profile()["stream_collide"] == (0.0, 0)


def run_ml(profile):
    ext, L = (128, 128, 128), 3
    pos = wl.particle_cloud(128, count=20000, seed=9, box=(0.25, 0.4, 0.25), y0_frac=0.2)
    with hl.Lattice(ext, levels=L, tau=0.9, periodic=(True, False, True), storage="f32") as lat:
        lat.set_profiling(profile)
        lat.rebuild_from_particles(pos)
        lat.deposit_particles(pos)
        lat.step(8)  # two coarse steps
        p = lat.profile()
        # level l takes 2^(L-1-l) steps per coarse step; a level without blocks launches nothing
        steps = 2 * sum(2 ** (L - 1 - l) for l in range(L) if lat.num_blocks(l) > 0)
        return p, steps, [lat.read_moments(level=l, dtype=np.float32) for l in range(L)]


def test_multilevel_profile_and_results_unchanged():
    p, steps, on = run_ml(True)
    _, _, off = run_ml(False)
    for a, b in zip(on, off):
        assert np.array_equal(a, b)
    assert p["stream_collide"][1] == steps
    assert p["down"][1] > 0 and p["up"][1] > 0
    assert p["rebuild"][1] == 1 and p["deposit"][1] == 1
    assert all(ms > 0 for ms, c in p.values() if c > 0)
