"""Batches of independent periodic domains (hlbm_batch_*) against the oracle.

* FP32 batch of uneven domains (including a single 8^3 block that wraps onto
  itself): every domain against the FP64 oracle, 1e-5 per step of the row scale;
* every launch strategy (one launch, graph, per-domain, persistent, persistent
  graph) gives bit-identical FP16-scaled results over 70 steps (two refits);
* a domain of a batch equals the same domain run as its own lattice, bit for
  bit, in FP32 and FP16-scaled storage (its scales are its own);
* FP16-scaled TGV domains of very different amplitudes against the oracle
  across a refit: per-domain scales keep each domain's relative error;
* the autotuner returns a valid mode and restores the state;
* the full 64-domain batch of the bench, one step, sampled nodes against
  single-node oracle updates.
"""
import numpy as np
import pytest
import torch

from oracle import single_level as sl
from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl
from tests.helpers import rel_err, row_scales

pytestmark = pytest.mark.gpu

RP_TOL = {"f16s": 8 * 2.0 ** -11, "bf16s": 8 * 2.0 ** -8}


def shape_of(extent):
    return (extent[2], extent[1], extent[0])


def fill(batch, fields):
    starts = []
    for d, M in enumerate(fields):
        batch.write_moments(d, hl.dense_to_blocks(M))
        starts.append(hl.blocks_to_dense(batch.read_moments(d), M.shape[1:]))
    return starts


def read_all(batch, domains):
    return [hl.blocks_to_dense(batch.read_moments(d), shape_of(e)) for d, (e, _) in enumerate(domains)]


def test_fp32_uneven_domains_match_oracle():
    domains = [((16, 16, 16), 0.6), ((32, 16, 24), 0.8), ((8, 8, 8), 0.55), ((24, 8, 16), 0.7)]
    fields = [wl.random_field(shape_of(e), 200 + d, du=0.03) for d, (e, _) in enumerate(domains)]
    steps = 3
    with hl.Batch(domains, storage="f32") as b:
        assert b.num_blocks() == sum(e[0] * e[1] * e[2] // 512 for e, _ in domains)
        starts = fill(b, fields)
        b.step(steps)
        got = read_all(b, domains)
    for d, (e, tau) in enumerate(domains):
        ref = sl.run(torch.tensor(starts[d]), steps, tau).numpy()
        err = rel_err(got[d], ref, row_scales(ref, 0.02))
        assert err.max() < steps * 1e-5, (d, err)


def batch_result(domains, fields, storage, mode, steps):
    with hl.Batch(domains, storage=storage) as b:
        b.set_mode(mode)
        fill(b, fields)
        b.step(steps)
        return read_all(b, domains)


def test_all_launch_strategies_agree_bitwise():
    rng = np.random.default_rng(7)
    domains = [((8 * int(rng.integers(1, 5)), 8 * int(rng.integers(1, 5)), 8 * int(rng.integers(1, 5))),
                float(rng.uniform(0.52, 0.8))) for _ in range(7)]
    fields = [wl.random_field(shape_of(e), 300 + d, du=float(rng.uniform(0.01, 0.08)))
              for d, (e, _) in enumerate(domains)]
    modes = [hl.BATCH_ONE_LAUNCH, hl.BATCH_GRAPH, hl.BATCH_PER_DOMAIN, hl.BATCH_PERSISTENT, hl.BATCH_PERSISTENT_GRAPH]
    base = batch_result(domains, fields, "f16s", modes[0], 70)
    for mode in modes[1:]:
        other = batch_result(domains, fields, "f16s", mode, 70)
        for d in range(len(domains)):
            assert np.array_equal(base[d], other[d]), (mode, d)


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_batch_domain_equals_own_lattice(storage):
    domains = [((16, 24, 8), 0.65), ((32, 32, 32), 0.58), ((8, 16, 8), 0.75)]
    fields = [wl.taylor_green_3d(32, 0.05) if e == (32, 32, 32) else wl.random_field(shape_of(e), 400 + d, du=0.02)
              for d, (e, _) in enumerate(domains)]
    got = batch_result(domains, fields, storage, hl.BATCH_GRAPH, 40)
    for d, (e, tau) in enumerate(domains):
        with hl.Lattice(e, tau=tau, storage=storage) as lat:
            lat.set_dense()
            lat.write_moments(hl.dense_to_blocks(fields[d]))
            lat.step(40)
            own = hl.blocks_to_dense(lat.read_moments(), shape_of(e))
        assert np.array_equal(got[d], own), d


def test_fp16_domains_of_different_amplitude_against_oracle():
    """Two 32^3 TGV domains, U0 = 0.08 and 0.002, 40 steps (a refit after 32):
    each against the FP64 oracle relative to its own amplitude."""
    domains = [((32, 32, 32), 0.6), ((32, 32, 32), 0.7)]
    amps = [0.08, 0.002]
    fields = [wl.taylor_green_3d(32, u) for u in amps]
    with hl.Batch(domains, storage="f16s") as b:
        starts = fill(b, fields)
        b.step(40)
        got = read_all(b, domains)
    for d, (e, tau) in enumerate(domains):
        ref = sl.run(torch.tensor(starts[d]), 40, tau).numpy()
        err = rel_err(got[d], ref, row_scales(ref, amps[d]))
        print("FP16 batch domain %d (U0 %.3f), 40 steps: max error / row scale (rho, u) %.3e" % (d, amps[d], err[:4].max()))
        assert err[:4].max() < 40 * RP_TOL["f16s"] / 4, (d, err)


def test_autotune_restores_state():
    domains = [((32, 32, 32), 0.6), ((48, 48, 48), 0.7), ((16, 16, 16), 0.55)]
    fields = [wl.taylor_green_3d(e[0], 0.05) for e, _ in domains]
    with hl.Batch(domains, storage="f16s") as b:
        fill(b, fields)
        b.step(5)
        before = read_all(b, domains)
        mode, ms = b.autotune(64)
        after = read_all(b, domains)
        assert mode in range(5) and all(t > 0 for t in ms)
        assert ms[mode] == min(ms)
        for d in range(len(domains)):
            assert np.array_equal(before[d], after[d])
        # stepping on from the restored state matches a fresh run of 5 + 33 steps
        b.step(33)
        cont = read_all(b, domains)
    fresh = batch_result(domains, fields, "f16s", hl.BATCH_ONE_LAUNCH, 38)
    for d in range(len(domains)):
        assert np.array_equal(cont[d], fresh[d])


def test_full_batch_sampled_nodes_one_step():
    """The 64-domain FP16-scaled batch of the bench (edges 32..128): one step,
    sampled nodes of four domains against single-node oracle updates from the
    decoded start state."""
    from tests.helpers import oracle_node_update
    doms = wl.batch_domains()
    domains = [((e, e, e), t) for e, _, t in doms]
    pick = [0, 21, 42, 63]
    with hl.Batch(domains, storage="f16s") as b:
        starts = {}
        for d, (e, u0, _) in enumerate(doms):
            M = wl.taylor_green_3d(e, u0).astype(np.float32)
            b.write_moments(d, torch.tensor(hl.dense_to_blocks(M), device="cuda"))
        for d in pick:
            e = doms[d][0]
            starts[d] = hl.blocks_to_dense(b.read_moments(d), (e, e, e))
        b.set_mode(hl.BATCH_GRAPH)
        b.step(1)
        got = {d: hl.blocks_to_dense(b.read_moments(d), (doms[d][0],) * 3) for d in pick}
    rng = np.random.default_rng(17)
    for d in pick:
        e, u0, tau = doms[d]
        nodes = [tuple(int(v) for v in rng.integers(0, e, 3)) for _ in range(6)] + [(0, 0, 0), (e - 1, e - 1, e - 1)]
        ref = oracle_node_update(starts[d], nodes, tau, (True, True, True))
        g = np.stack([got[d][:, z, y, x] for (x, y, z) in nodes], axis=1)
        err = rel_err(g, ref, row_scales(ref, u0))
        assert err.max() < RP_TOL["f16s"], (d, err)
