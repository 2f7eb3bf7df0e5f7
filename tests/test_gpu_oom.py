"""Out-of-memory paths of the C ABI, simulated on the host.

hlbm_inject_alloc_failure(k) makes the device allocation after k more
successful ones fail, as a real out-of-memory would.  Each test walks k from 0
until a call sequence runs through without the injected failure, and checks
at every failure point that

* the failing call returns E_OOM (nothing else, no CUDA error);
* the handle keeps the state the header promises (the previous hierarchy and
  moments after a failed rebuild, no blocks after a failed set-up, no
  recording after a failed forward_record, the state after a failed
  autotune of a batch);
* with the injection cleared, the same calls on the same handle give the same
  results as a run that never failed, and the handle is destroyed cleanly.
"""
import numpy as np
import pytest
import torch

from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl
from tests.helpers import ml_adjoint_case

pytestmark = pytest.mark.gpu

K_MAX = 200   # more allocations than any sequence below makes


@pytest.fixture(autouse=True)
def _clear_injection():
    hl.inject_alloc_failure(-1)
    yield
    hl.inject_alloc_failure(-1)


def walk(run):
    """run(k) injects a failure after k allocations and returns True once the
    sequence ran through without meeting it; returns the number of failure
    points seen."""
    for k in range(K_MAX):
        if run(k):
            hl.inject_alloc_failure(-1)
            return k
    raise AssertionError("the sequence never ran through")


def expect_oom(call):
    """Run call(); True if it ran, False if it failed with E_OOM (any other
    failure raises)."""
    try:
        call()
        return True
    except hl.HlbmError as e:
        assert e.code == hl.E_OOM, e
        return False


def single_level_sequence(lat, F, eps):
    lat.set_dense()
    lat.write_moments(hl.dense_to_blocks(wl.random_field((16, 16, 32), 5, du=0.01)))
    lat.set_force(F, eps)
    lat.step(3)
    return lat.read_moments()


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_single_level_set_up_and_steps_fail_cleanly(storage):
    nb = 2 * 2 * 4
    g = torch.Generator().manual_seed(3)
    F = (torch.randn((nb, 3, 512), generator=g) * 1e-5).cuda()
    eps = (0.8 + 0.2 * torch.rand((nb, 512), generator=g)).cuda()
    with hl.Lattice((32, 16, 16), tau=0.7, periodic=(True, True, True), storage=storage) as ref:
        want = single_level_sequence(ref, F, eps)

    def run(k):
        with hl.Lattice((32, 16, 16), tau=0.7, periodic=(True, True, True), storage=storage) as lat:
            hl.inject_alloc_failure(k)
            ran = expect_oom(lambda: single_level_sequence(lat, F, eps))
            hl.inject_alloc_failure(-1)
            if not ran:
                got = single_level_sequence(lat, F, eps)   # same handle, injection cleared
                assert np.array_equal(got, want), k
            return ran

    assert walk(run) >= 5


def test_failed_set_dense_leaves_no_blocks():
    with hl.Lattice((32, 16, 16), tau=0.7, storage="f32") as lat:
        lat.set_dense()
        lat.step(1)
        hl.inject_alloc_failure(1)    # the neighbour table goes through, a moment buffer fails
        with pytest.raises(hl.HlbmError) as ei:
            lat.set_dense()
        assert ei.value.code == hl.E_OOM
        hl.inject_alloc_failure(-1)
        for call in (lambda: lat.step(1), lambda: lat.read_moments(), lambda: lat.reduce()):
            with pytest.raises(hl.HlbmError) as ei:
                call()
            assert ei.value.code == hl.E_BAD_STATE
        lat.set_dense()
        lat.step(1)


def test_failed_rebuild_keeps_previous_hierarchy():
    c = ml_adjoint_case("three_level_wall")
    ext, L = c["ext"], c["L"]
    z, y, x = np.nonzero(c["O0"])
    first = np.stack([x, y, z], axis=1)
    second = first + np.array([1, 0, 1])       # the refined patch moves by one block

    def prepared():
        lat = hl.Lattice(ext, levels=L, tau=c["tau0"], periodic=c["periodic"], storage="f32")
        lat.set_fine_blocks(first)
        for l in range(L):
            cl, _ = lat.blocks(l)
            lat.write_moments(hl.dense_to_blocks(c["M0"][l], cl), level=l)
        lat.step(4)
        return lat

    with prepared() as ref:
        ref.set_fine_blocks(second)
        ref.step(4)
        want = [ref.read_moments(level=l) for l in range(L)]
        want_blocks = [ref.blocks(l)[0] for l in range(L)]

    with prepared() as lat:
        before = [lat.read_moments(level=l) for l in range(L)]
        before_blocks = [lat.blocks(l)[0] for l in range(L)]

        def run(k):
            hl.inject_alloc_failure(k)
            ran = expect_oom(lambda: lat.set_fine_blocks(second))
            hl.inject_alloc_failure(-1)
            if not ran:
                for l in range(L):
                    assert np.array_equal(lat.blocks(l)[0], before_blocks[l]), (k, l)
                    assert np.array_equal(lat.read_moments(level=l), before[l]), (k, l)
            return ran

        assert walk(run) >= 20
        lat.step(4)
        for l in range(L):
            assert np.array_equal(lat.blocks(l)[0], want_blocks[l]), l
            assert np.array_equal(lat.read_moments(level=l), want[l]), l


def test_failed_rebuild_from_particles_keeps_previous_hierarchy():
    ext = (64, 64, 64)
    rng = np.random.default_rng(4)
    a = (rng.random((3000, 3)) * [16, 16, 16] + [8, 8, 8]).astype(np.float32)
    b = a + np.float32(24.0)
    with hl.Lattice(ext, levels=2, tau=0.8, periodic=(True, True, True), storage="f32") as lat:
        lat.rebuild_from_particles(a)
        lat.step(2)
        before = [lat.read_moments(level=l) for l in range(2)]
        before_blocks = [lat.blocks(l)[0] for l in range(2)]

        def run(k):
            hl.inject_alloc_failure(k)
            ran = expect_oom(lambda: lat.rebuild_from_particles(b))
            hl.inject_alloc_failure(-1)
            if not ran:
                for l in range(2):
                    assert np.array_equal(lat.blocks(l)[0], before_blocks[l]), (k, l)
                    assert np.array_equal(lat.read_moments(level=l), before[l]), (k, l)
            return ran

        assert walk(run) >= 20
        lat.step(2)


@pytest.mark.parametrize("multilevel", [False, True])
def test_failed_record_and_adjoint_recover(multilevel):
    if multilevel:
        c = ml_adjoint_case("two_level")
        lat = hl.Lattice(c["ext"], levels=c["L"], tau=c["tau0"], periodic=c["periodic"], storage="f32")
        z, y, x = np.nonzero(c["O0"])
        lat.set_fine_blocks(np.stack([x, y, z], axis=1))
        n_lv = c["L"]
    else:
        lat = hl.Lattice((32, 16, 16), tau=0.8, periodic=(True, True, True), storage="f32")
        lat.set_dense()
        n_lv = 1
    with lat:
        coords = [lat.blocks(l)[0] for l in range(n_lv)]
        g = torch.Generator().manual_seed(9)
        M0 = c["M0"] if multilevel else [wl.random_field((16, 16, 32), 9)]
        for l in range(n_lv):
            lat.write_moments(hl.dense_to_blocks(M0[l], coords[l]), level=l)
        M_start = [lat.read_moments(level=l) for l in range(n_lv)]
        F = (torch.randn((len(coords[0]), 3, 512), generator=g) * 1e-5).cuda()
        lat.set_force(F)
        per = 1 << (n_lv - 1)
        n_steps, ckpt = 4 * per, 2 * per
        W = torch.randn((sum(len(cl) for cl in coords), 10, 512), generator=g).cuda()

        def restart():
            for l in range(n_lv):
                lat.write_moments(M_start[l], level=l)

        restart()
        lat.forward_record(n_steps, ckpt)
        want = lat.adjoint(W, torch.empty_like(F)).cpu().numpy()
        assert np.isfinite(want).all() and np.abs(want).max() > 0

        def run_record(k):
            restart()
            hl.inject_alloc_failure(k)
            ran = expect_oom(lambda: lat.forward_record(n_steps, ckpt))
            hl.inject_alloc_failure(-1)
            if not ran:
                with pytest.raises(hl.HlbmError) as ei:     # nothing was recorded
                    lat.adjoint(W, torch.empty_like(F))
                assert ei.value.code == hl.E_BAD_STATE
            return ran

        walk(run_record)

        def run_adjoint(k):
            hl.inject_alloc_failure(k)
            dF = torch.empty_like(F)
            ran = expect_oom(lambda: lat.adjoint(W, dF))
            hl.inject_alloc_failure(-1)
            if not ran:                                      # the recording is kept: retry
                dF = lat.adjoint(W, torch.empty_like(F))
            got = dF.cpu().numpy()
            err = np.abs(got - want).max() / np.abs(want).max()
            assert err < 1e-6, (k, err)
            return ran

        assert walk(run_adjoint) >= 5


def test_batch_create_steps_and_autotune_fail_cleanly():
    domains = [((16, 16, 16), 0.6), ((32, 16, 24), 0.8), ((8, 8, 8), 0.55)]
    fields = [hl.dense_to_blocks(wl.random_field((e[2], e[1], e[0]), 300 + d, du=0.03))
              for d, (e, _) in enumerate(domains)]

    def sequence(b):
        b.set_mode(hl.BATCH_PERSISTENT)
        for d, M in enumerate(fields):
            b.write_moments(d, M)
        b.step(3)
        return [b.read_moments(d) for d in range(len(domains))]

    with hl.Batch(domains, storage="f16s") as b:
        want = sequence(b)

    def run(k):
        hl.inject_alloc_failure(k)
        try:
            b = hl.Batch(domains, storage="f16s")
        except hl.HlbmError as e:           # a failed create frees what it allocated
            assert e.code == hl.E_OOM, e
            return False
        with b:
            ran = expect_oom(lambda: sequence(b))
            hl.inject_alloc_failure(-1)
            got = sequence(b)               # same handle, injection cleared
            assert all(np.array_equal(g, w) for g, w in zip(got, want)), k
            if ran:                         # the autotuner's state copy fails: nothing changes
                hl.inject_alloc_failure(0)
                with pytest.raises(hl.HlbmError) as ei:
                    b.autotune(8)
                assert ei.value.code == hl.E_OOM
                hl.inject_alloc_failure(-1)
                assert all(np.array_equal(b.read_moments(d), w) for d, w in enumerate(want))
        return ran

    assert walk(run) >= 8
