"""Throughput of the moment-encoded lattice Boltzmann hot path on GB300.

Default workload: the dense 256^3 force-driven duct (periodic x, half-way
bounce-back walls in y and z, 8^3 blocks, FP32 moments, tau = 0.55, body force
1e-6 along x).  One step = one fused pull-stream + collide launch over all
32,768 blocks.  The moment buffers (671 MB each) are far larger than the
129 MB L2, so no flush is needed between steps.

Printed JSON keys: value = fine-equivalent MLUPS (nodes x steps / s, device
time), roofline = the stream-collide kernel's algorithmic bytes (read + write
of 10 FP32 moments per node = 80 B) / its CUDA-event time against the measured
HBM copy bandwidth, e2e = the same metric through the C ABI with host buffers
(upload of the initial state, the steps, download of the final state and the
FP64 reductions, all timed), cpu_baseline = the FP64 CPU oracle on a bounded
sample of the same duct.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs an independent replica (the single domain does
not shard): value = all ranks' node updates / the slowest rank.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine-equiv MLUPS and % HBM roofline per step; adjoint/forward time ratio"
BYTES_PER_NODE_F32 = 80.0
KERNEL = "k_stream_collide_f2<float>"
# DRAM bytes (read + write) per launch of KERNEL from one ncu capture of the
# 192^3 duct, scaled by nodes to 256^3 (profiles/stream_collide_f2_duct192.md);
# set to None whenever the kernel changes after that capture.
TRAFFIC_PER_NODE = (289.211648e6 + 242.613504e6) / 192 ** 3
# FP32 operations per node update of KERNEL (ncu thread-level counts of FADD,
# FMUL, FFMA and their packed forms on the 192^3 duct, profiles/
# stream_collide_f2_duct192.md; FMA = 2); None when not measured for the
# current kernel.
FLOP_PER_NODE = 531.3


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def fp32_sgemm_tflops(n=8192, reps=10):
    """FP32 CUDA-core rate of this GPU: cuBLAS SGEMM with TF32 off (2 n^3 flop each)."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        for _ in range(3):
            c = a @ b
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            c = a @ b
        ev[1].record()
        ev[1].synchronize()
        del a, b, c
        return 2.0 * n ** 3 * reps / (ev[0].elapsed_time(ev[1]) / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank timings (seconds) over all ranks."""
    if world <= 1:
        return list(values)
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_mlups(nodes, steps, world, seconds):
    """Whole-job throughput of independent replicas: every rank advances its own
    copy of the workload, so the job updates world * nodes * steps nodes in the
    slowest rank's time."""
    return world * nodes * steps / seconds / 1e6


STORAGE_BYTES = {"f32": BYTES_PER_NODE_F32, "f16s": 40.0, "bf16s": 40.0}
STORAGE_KERNEL = {"f32": KERNEL, "f16s": "k_stream_collide_f2<__half>", "bf16s": "k_stream_collide_f2<__nv_bfloat16>"}


def duct_lattice(hl, n, stream, storage="f32"):
    lat = hl.Lattice((n, n, n), tau=0.55, periodic=(True, False, False), storage=storage, stream=stream)
    lat.set_dense()
    lat.set_uniform_force(1e-6, 0.0, 0.0)
    return lat


def run_gpu(args, rank, world):
    import torch
    from paper_2603_14982_gb300 import build as B
    from paper_2603_14982_gb300 import homelbm as hl
    from paper_2603_14982_gb300 import workloads as wl

    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    n = args.n
    nodes = n ** 3
    lat = duct_lattice(hl, n, stream.cuda_stream, args.storage)
    lat.cfg.device = dev
    # --- device-resident timing
    for _ in range(args.warmup):
        lat.step(1)
    lat.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        lat.step(args.steps)
        ev[1].record(stream)
    ev[1].synchronize()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[1])
    red = lat.reduce()
    lat.close()
    # --- end to end through the C ABI with host buffers
    M0 = hl.dense_to_blocks(wl.rest_field((n, n, n)).astype(np.float32))
    host_in = torch.from_numpy(M0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    lat = duct_lattice(hl, n, stream.cuda_stream, args.storage)
    lat.write_moments(host_in.numpy())
    lat.step(2)
    lat.synchronize()
    t0 = time.perf_counter()
    lat.write_moments(host_in.numpy())
    lat.step(args.steps)
    lat.read_moments(host_out.numpy())
    red_e2e = lat.reduce()
    t_e2e = time.perf_counter() - t0
    lat.close()
    t_dev, t_e2e = max_over_ranks([ms / 1e3, t_e2e], world, "cuda")
    extras = None
    if not args.no_extras and world == 1:
        extras = bench_extras(hl, wl)
    res = {
        "extras": extras,
        "ms_per_step": 1e3 * t_dev / args.steps,
        "value": job_mlups(nodes, args.steps, world, t_dev),
        "e2e_value": job_mlups(nodes, args.steps, world, t_e2e),
        "clocks": clk,
        "mass": red[0],
        "e2e_bytes": M0.nbytes,
        "finite": bool(np.isfinite(red_e2e[0])),
    }
    return res


def timed(stream, fn):
    """Device time (ms) of fn() on a stream, bracketed by synchronizes."""
    import torch
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    fn()
    ev[1].record(stream)
    ev[1].synchronize()
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1])


def bench_batched(hl, wl, stream, steps=200):
    """64 uneven periodic Taylor-Green domains (edges from {32,48,64,96,128},
    U0 in [0.01, 0.08], tau in [0.52, 0.8], seeded), FP16-scaled storage: the
    autotuned batch against one launch per domain, and the FP32 batch."""
    import torch
    doms = wl.batch_domains()
    domains = [((e, e, e), t) for e, _, t in doms]
    nodes = sum(e ** 3 for e, _, _ in doms)
    init = [torch.tensor(hl.dense_to_blocks(wl.taylor_green_3d(e, u0).astype(np.float32)), device="cuda")
            for e, u0, _ in doms]
    out = {"domains": len(doms), "nodes": nodes, "steps": steps}
    finals = {}
    names = ["one_launch", "graph", "per_domain", "persistent", "persistent_graph"]
    for storage in ("f16s", "f32"):
        with hl.Batch(domains, storage=storage, stream=stream.cuda_stream) as b:
            for d in range(len(doms)):
                b.write_moments(d, init[d])
            mode, trial_ms = b.autotune(64)
            ms = timed(stream, lambda: b.step(steps))
            rec = {"mode": names[mode], "autotune_ms_per_step": dict(zip(names, [round(t, 4) for t in trial_ms])),
                   "ms_per_step": round(ms / steps, 4), "mlups": round(nodes * steps / ms / 1e3, 1),
                   "bytes_per_node": 40.0 if storage == "f16s" else 80.0}
            rec["hbm_gbs"] = round(rec["bytes_per_node"] * nodes * steps / ms / 1e6, 1)
            if storage == "f16s":
                b.set_mode(hl.BATCH_PER_DOMAIN)
                ms_pd = timed(stream, lambda: b.step(steps))
                rec["per_domain_ms_per_step"] = round(ms_pd / steps, 4)
                rec["per_domain_mlups"] = round(nodes * steps / ms_pd / 1e3, 1)
                rec["speedup_vs_per_domain"] = round(ms_pd / ms, 3)
                b.set_mode(mode)
            # accuracy: the same `steps` steps from the initial state, first eight domains
            for d in range(len(doms)):
                b.write_moments(d, init[d])
            b.step(steps)
            finals[storage] = [b.read_moments(d, torch.empty((b.num_blocks(d), 10, 512), dtype=torch.float32,
                                                             device="cuda"))[:, 1:4].clone() for d in range(8)]
            out[storage] = rec
    out["f16s_vs_f32_max_du_over_U0"] = max(float((finals["f16s"][d] - finals["f32"][d]).abs().max() / doms[d][1])
                                            for d in range(8))
    return out


def bench_adjoint(hl, wl, stream, n=128, steps=200, ckpt=20):
    """Forward vs checkpointed adjoint on the 128^3 channel with the central 16^3 obstacle."""
    import torch
    shape = (n, n, n)
    solid = wl.obstacle_mask(n).astype(np.uint8)
    F = torch.tensor(hl.dense_to_blocks(wl.noisy_force(shape).astype(np.float32)), device="cuda")
    M0 = torch.tensor(hl.dense_to_blocks(wl.rest_field(shape).astype(np.float32)), device="cuda")
    with hl.Lattice(shape, tau=0.55, periodic=(True, False, False), storage="f32", stream=stream.cuda_stream) as lat:
        lat.set_dense()
        lat.set_solid(solid)
        lat.set_force(F)
        lat.write_moments(M0)
        lat.step(20)
        lat.write_moments(M0)
        t_fwd = timed(stream, lambda: lat.step(steps))
        lam = torch.zeros((lat.num_blocks(0), 10, 512), dtype=torch.float32, device="cuda")
        lam[:, 1:4] = 1e-3
        dF = torch.empty((lat.num_blocks(0), 3, 512), dtype=torch.float32, device="cuda")
        # one untimed recording and adjoint first, as the forward had its warm-up
        # steps (the first calls also grow the memory pool by their buffers)
        lat.write_moments(M0)
        lat.forward_record(steps, ckpt)
        lat.adjoint(lam, dF)
        lat.write_moments(M0)
        t_rec = timed(stream, lambda: lat.forward_record(steps, ckpt))
        t_adj = timed(stream, lambda: lat.adjoint(lam, dF))
    return {"n": n, "steps": steps, "ckpt_every": ckpt, "forward_ms": round(t_fwd, 3),
            "forward_record_ms": round(t_rec, 3), "adjoint_ms": round(t_adj, 3),
            "adjoint_over_forward": round(t_adj / t_fwd, 3),
            "record_plus_adjoint_over_forward": round((t_rec + t_adj) / t_fwd, 3),
            "finite": bool(torch.isfinite(dF).all().item())}


def bench_ml_adjoint(hl, wl, stream, pos0, n=512, fine_steps=40, ckpt=8):
    """Forward vs checkpointed adjoint of the three-level advance (Algorithm 1
    with both transfers) on the n^3 fine-equivalent hierarchy of the falling
    cloud at its start, with its deposited drag and fluid fraction; FP32."""
    import torch
    L = 3
    with hl.Lattice((n, n, n), levels=L, tau=0.9, periodic=(True, False, True), storage="f32",
                    stream=stream.cuda_stream) as lat:
        lat.rebuild_from_particles(pos0)
        lat.deposit_particles(pos0)
        counts = [lat.num_blocks(l) for l in range(L)]
        start = [lat.read_moments(torch.empty((c, 10, 512), dtype=torch.float32, device="cuda"), level=l)
                 for l, c in enumerate(counts)]

        def reset():
            for l in range(L):
                lat.write_moments(start[l], level=l)

        lat.step(8)  # loads every kernel once
        reset()
        t_fwd = timed(stream, lambda: lat.step(fine_steps))
        lam = torch.zeros((sum(counts), 10, 512), dtype=torch.float32, device="cuda")
        lam[:, 1:4] = 1e-3
        dF = torch.empty((counts[0], 3, 512), dtype=torch.float32, device="cuda")
        # one untimed recording and adjoint first (warm-up; pool growth)
        reset()
        lat.forward_record(fine_steps, ckpt)
        lat.adjoint(lam, dF)
        reset()
        t_rec = timed(stream, lambda: lat.forward_record(fine_steps, ckpt))
        t_adj = timed(stream, lambda: lat.adjoint(lam, dF))
    return {"n": n, "levels": L, "fine_steps": fine_steps, "ckpt_every": ckpt, "blocks_per_level": counts,
            "forward_ms": round(t_fwd, 3), "forward_record_ms": round(t_rec, 3), "adjoint_ms": round(t_adj, 3),
            "adjoint_over_forward": round(t_adj / t_fwd, 3),
            "record_plus_adjoint_over_forward": round((t_rec + t_adj) / t_fwd, 3),
            "finite": bool(torch.isfinite(dF).all().item())}


def bench_sparse(hl, wl, stream, n=2048, L=4, coarse_steps=4, lookup=0):
    """Fine-equivalent throughput on the sparse n^3 tube-tree hierarchy (four
    levels, bounce-back walls on every face, uniform force 1e-6 along -y, FP32,
    static hierarchy): hierarchy build time, then coarse steps timed with CUDA
    events after one warm-up coarse step.  lookup: block lookup mode (0 dense
    slot tables, 1 spatial hash)."""
    import torch
    per = 2 ** (L - 1)
    coords = wl.tube_tree_blocks(n)
    with hl.Lattice((n, n, n), levels=L, tau=0.9, periodic=(False, False, False), storage="f32",
                    stream=stream.cuda_stream) as lat:
        lat.set_block_lookup(lookup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.set_fine_blocks(coords)
        lat.synchronize()
        t_build = time.perf_counter() - t0
        mode, table_bytes = lat.block_lookup()
        lat.set_uniform_force(0.0, -1e-6, 0.0)
        counts = [lat.num_blocks(l) for l in range(L)]
        lat.step(per)
        t = timed(stream, lambda: lat.step(per * coarse_steps))
        red = lat.reduce()
    updates = coarse_steps * sum(counts[l] * 512 * 2 ** (L - 1 - l) for l in range(L))
    fine_steps = per * coarse_steps
    peak, _ = measured_peaks()
    gbs = updates * 80.0 / (t / 1e3) / 1e9
    return {"n": n, "levels": L, "blocks_per_level": counts, "tree_blocks": int(len(coords)),
            "effective_over_actual": round(n ** 3 / (sum(counts) * 512), 1),
            "moment_bytes": int(sum(counts) * 512 * 40 * 2), "build_s": round(t_build, 3), "fine_steps": fine_steps,
            "ms_per_fine_step": round(t / fine_steps, 3),
            "mlups_fine_equiv": round(n ** 3 * fine_steps / (t / 1e3) / 1e6, 1),
            "actual_updates_per_s_M": round(updates / (t / 1e3) / 1e6, 1),
            "actual_gbs": round(gbs, 1), "actual_gbs_over_peak": round(gbs / peak, 4),
            "mass": float(red[0]), "finite": bool(np.isfinite(red[0])),
            "block_lookup": "hash" if mode == 1 else "slot tables", "lookup_table_bytes": int(table_bytes)}


def bench_multilevel(hl, wl, stream, storage, pos0, n=512, fine_steps=500, rebuild_every=10, drag_every=0,
                     profile=False):
    """Three-level lattice over an n^3 fine-equivalent domain driven by a falling
    particle cloud (pos0, device, not modified): rebuild at the first
    coarse-step boundary at least rebuild_every fine steps after the last one,
    deposit of eta / eps / drag every coarse step.  Fine-equivalent MLUPS over
    the whole loop (wall clock, everything on one stream; only the rebuilds,
    which read block counts back, wait for the device).  drag_every > 0: the
    coupled step (streaming only, live drag F = 1e-4 eta (v_p - u*) with the
    cloud's velocity v_p = (0, -1, 0), collision) every drag_every finest-level
    steps."""
    import torch
    L = 3
    per = 2 ** (L - 1)
    pos = pos0.clone()
    with hl.Lattice((n, n, n), levels=L, tau=0.9, periodic=(True, False, True), storage=storage,
                    stream=stream.cuda_stream) as lat:
        if drag_every:
            lat.set_drag(1e-4, (0.0, -1.0, 0.0), drag_every)
        lat.rebuild_from_particles(pos)
        lat.deposit_particles(pos)
        torch.cuda.synchronize()
        if profile:  # stream time per kernel class over the timed loop (CUDA events in the library)
            lat.set_profiling(True)
        t_reb = 0.0
        updates = 0
        updates0 = 0   # finest-level updates (they also read the force and fluid-fraction fields)
        since = 0
        rebuilds = 0
        counts = [lat.num_blocks(l) for l in range(L)]
        t0 = time.perf_counter()
        for k in range(fine_steps // per):
            lat.step(per)
            updates += sum(counts[l] * 512 * 2 ** (L - 1 - l) for l in range(L))
            updates0 += counts[0] * 512 * 2 ** (L - 1)
            since += per
            with torch.cuda.stream(stream):
                pos[:, 1] = torch.clamp(pos[:, 1] - per, min=0.5)
            if since >= rebuild_every:
                lat.synchronize()   # the rebuild waits for the device anyway; attribute only its own time
                t1 = time.perf_counter()
                lat.rebuild_from_particles(pos)
                t_reb += time.perf_counter() - t1
                counts = [lat.num_blocks(l) for l in range(L)]
                since = 0
                rebuilds += 1
            lat.deposit_particles(pos, moving=bool(k < fine_steps // per - 1), wait=False)
        lat.synchronize()
        t_tot = time.perf_counter() - t0
        prof = None
        if profile:
            prof = {k: {"ms": round(v[0], 3), "spans": v[1]} for k, v in lat.profile().items()}
            lat.set_profiling(False)
        # deposit cost alone (input preparation, not part of the method)
        t_dep = timed(stream, lambda: [lat.deposit_particles(pos, wait=False) for _ in range(10)]) / 10
        red = lat.reduce()
        moms = [lat.read_moments(torch.empty((lat.num_blocks(l), 10, 512), dtype=torch.float32, device="cuda"),
                                 level=l) for l in range(L)]
    bpn = 80.0 if storage == "f32" else 40.0
    actual_gbs = (updates * bpn + updates0 * 16.0) / t_tot / 1e9
    peak, _ = measured_peaks()
    return {"storage": storage, "fine_steps": fine_steps, "rebuilds": rebuilds,
            "actual_gbs": round(actual_gbs, 1), "actual_gbs_over_peak": round(actual_gbs / peak, 4),
            "mlups_fine_equiv": round(n ** 3 * fine_steps / t_tot / 1e6, 1),
            "actual_updates_per_s_M": round(updates / t_tot / 1e6, 1),
            "total_s": round(t_tot, 4), "rebuild_s": round(t_reb, 4), "rebuild_ms_each": round(1e3 * t_reb / rebuilds, 3),
            "deposit_ms_each": round(t_dep, 4),
            "blocks_per_level_end": counts, "mass_rel_drift": float(red[0] / n ** 3 - 1.0),
            "finite": bool(np.isfinite(red[0])), **({"profile": prof} if prof is not None else {})}, moms


def bench_open_dune(hl, wl, stream, open_faces=True, extent=(512, 128, 256), fine_steps=64):
    """Three-level channel over a resting sand heap (a dune-shaped seeded
    particle cloud on the floor): logarithmic inlet at x-, convective outflow
    at x+ and on the top face, bounce-back floor, periodic z; the hierarchy
    from the heap, the fluid fraction deposited from it.  With
    open_faces=False the same lattice is periodic in x (the open faces'
    cost is the difference).  Device time of fine_steps fine steps (CUDA
    events), then the open-face updates' share from the library's profile."""
    import torch
    L, per = 3, 4
    pos = torch.tensor(wl.sand_heap(extent), device="cuda")
    periodic = (not open_faces, False, True)
    with hl.Lattice(extent, levels=L, tau=0.9, periodic=periodic, storage="f32", stream=stream.cuda_stream) as lat:
        if open_faces:
            lat.set_open_faces([hl.FACE_INLET, hl.FACE_OUTFLOW, hl.FACE_CLOSED, hl.FACE_OUTFLOW,
                                hl.FACE_CLOSED, hl.FACE_CLOSED], u0=0.005, beta=1.0, h0=0.0, profile_axis=1)
        lat.rebuild_from_particles(pos)
        lat.deposit_particles(pos, moving=False)
        counts = [lat.num_blocks(l) for l in range(L)]
        lat.step(2 * per)
        ms = timed(stream, lambda: lat.step(fine_steps))
        lat.set_profiling(True)
        lat.step(fine_steps)
        prof = lat.profile()
        lat.set_profiling(False)
        red = lat.reduce()
    updates = sum(counts[l] * 512 * 2 ** (L - 1 - l) for l in range(L)) * fine_steps // per
    updates0 = counts[0] * 512 * fine_steps
    actual_gbs = (updates * 80.0 + updates0 * 16.0) / (ms / 1e3) / 1e9
    peak, _ = measured_peaks()
    prof_total = sum(v[0] for v in prof.values())
    return {"extent": list(extent), "open_faces": bool(open_faces), "levels": L, "blocks_per_level": counts,
            "fine_steps": fine_steps, "ms_per_fine_step": round(ms / fine_steps, 4),
            "mlups_fine_equiv": round(extent[0] * extent[1] * extent[2] * fine_steps / ms / 1e3, 1),
            "actual_gbs": round(actual_gbs, 1), "actual_gbs_over_peak": round(actual_gbs / peak, 4),
            "open_face_share": round(prof["open_faces"][0] / prof_total, 4) if prof_total > 0 else 0.0,
            "mass": float(red[0]), "finite": bool(np.isfinite(red[0]))}


def bench_duct_storage(hl, stream, storage, n=256, steps=100, warmup=10):
    """The same duct in another moment storage: device time per step, MLUPS and
    the algorithmic bytes (40 per node in FP16/BF16-scaled storage) over the
    measured HBM peak."""
    lat = duct_lattice(hl, n, stream.cuda_stream, storage)
    try:
        lat.step(warmup)
        ms = timed(stream, lambda: lat.step(steps)) / steps
        mass = lat.reduce()[0]
    finally:
        lat.close()
    peak, _ = measured_peaks()
    bpn = STORAGE_BYTES[storage]
    return {"storage": storage, "ms_per_step": round(ms, 5), "mlups": round(n ** 3 / ms / 1e3, 1),
            "bytes_per_node": bpn, "frac": round(n ** 3 * bpn / (ms / 1e3) / 1e9 / peak, 4),
            "mass_rel_drift": float(mass / n ** 3 - 1.0)}


def bench_extras(hl, wl):
    import torch
    stream = torch.cuda.Stream()
    out = {"duct_f16s": bench_duct_storage(hl, stream, "f16s"), "duct_bf16s": bench_duct_storage(hl, stream, "bf16s"),
           "c5_batched": bench_batched(hl, wl, stream), "c4_adjoint": bench_adjoint(hl, wl, stream),
           "fp32_sgemm_tflops": round(fp32_sgemm_tflops(), 1)}
    ml = {}
    ref = None
    pos0 = torch.tensor(wl.particle_cloud(512), device="cuda")
    for storage in ("f32", "f16s", "bf16s"):
        bench_multilevel(hl, wl, stream, storage, pos0, fine_steps=48)   # warm-up: loads every kernel once
        rec, moms = bench_multilevel(hl, wl, stream, storage, pos0)
        if storage == "f32":
            ref = moms
        else:
            du = max(float((a[:, 1:4] - b[:, 1:4]).abs().max()) for a, b in zip(moms, ref))
            umax = max(float(b[:, 1:4].abs().max()) for b in ref)
            rec["max_du_vs_f32_over_umax"] = du / max(umax, 1e-30)
        ml[storage] = rec
    out["c3_multilevel"] = ml
    bench_multilevel(hl, wl, stream, "f32", pos0, fine_steps=48, drag_every=4)
    rec, _ = bench_multilevel(hl, wl, stream, "f32", pos0, drag_every=4)
    rec["drag_every"] = 4
    rec["mlups_vs_uncoupled"] = round(rec["mlups_fine_equiv"] / ml["f32"]["mlups_fine_equiv"], 3)
    out["c3_coupled"] = rec
    out["c3_adjoint"] = bench_ml_adjoint(hl, wl, stream, pos0)
    dune = bench_open_dune(hl, wl, stream)
    closed = bench_open_dune(hl, wl, stream, open_faces=False)
    dune["ms_per_fine_step_periodic_x"] = closed["ms_per_fine_step"]
    out["f3_open_dune"] = dune
    out["sparse_tree_2048"] = bench_sparse(hl, wl, stream)
    hashed = bench_sparse(hl, wl, stream, lookup=1)
    out["sparse_tree_2048_hash"] = {k: hashed[k] for k in ("ms_per_fine_step", "mlups_fine_equiv", "build_s",
                                                           "block_lookup", "lookup_table_bytes", "mass")}
    return out


def cpu_oracle_sample(n_sample=64, steps=12, threads=None):
    """The FP64 CPU oracle on an n_sample^3 duct of the same kind (bounded sample),
    on `threads` host threads (default: torch's, normally every core)."""
    import torch
    from oracle import single_level as sl
    from paper_2603_14982_gb300 import workloads as wl

    prev = torch.get_num_threads()
    if threads is not None:
        torch.set_num_threads(threads)
    try:
        M = torch.tensor(wl.rest_field((n_sample,) * 3))
        blocked = sl.blocked_sources(M.shape[1:], (True, False, False))
        sl.step(M, 0.55, force=(1e-6, 0, 0), periodic=(True, False, False), blocked=blocked)
        t0 = time.perf_counter()
        for _ in range(steps):
            M = sl.step(M, 0.55, force=(1e-6, 0, 0), periodic=(True, False, False), blocked=blocked)
        dt = time.perf_counter() - t0
        used = torch.get_num_threads()
    finally:
        torch.set_num_threads(prev)
    return {"value": n_sample ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": used,
            "kind": "oracle", "sample": "%d^3 duct of the same kind, %d steps, FP64 torch CPU, %d threads, %.1f s" %
            (n_sample, steps, used, dt)}


def cpu_baseline():
    """The oracle on every host core and on one, with the host's core count."""
    allc = cpu_oracle_sample(128, 16)
    one = cpu_oracle_sample(64, 6, threads=1)
    allc["single_thread"] = {"value": one["value"], "unit": "MLUPS", "cores": 1, "sample": one["sample"]}
    allc["nproc"] = os.cpu_count()
    return allc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16s", "bf16s"],
                    help="moment storage of the duct (the metric's configuration is f32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the multi-level, adjoint and batched workloads")
    ap.add_argument("--only", choices=["multilevel", "adjoint", "batched", "ml_adjoint", "sparse", "open_dune"],
                    help="run one secondary workload alone and print its JSON (profiling runs)")
    ap.add_argument("--profile", action="store_true",
                    help="with --only multilevel: stream time per kernel class from the library's CUDA events")
    ap.add_argument("--adj-steps", type=int, default=200)
    ap.add_argument("--adj-ckpt", type=int, default=20)
    args = ap.parse_args()
    if args.only:
        import torch
        from paper_2603_14982_gb300 import build as B
        from paper_2603_14982_gb300 import homelbm as hl
        from paper_2603_14982_gb300 import workloads as wl
        B.build()
        stream = torch.cuda.Stream()
        if args.only == "adjoint":
            res = bench_adjoint(hl, wl, stream, steps=args.adj_steps, ckpt=args.adj_ckpt)
        elif args.only == "batched":
            res = bench_batched(hl, wl, stream)
        elif args.only == "sparse":
            res = bench_sparse(hl, wl, stream)
        elif args.only == "ml_adjoint":
            res = bench_ml_adjoint(hl, wl, stream, torch.tensor(wl.particle_cloud(512), device="cuda"))
        elif args.only == "open_dune":
            res = bench_open_dune(hl, wl, stream)
            res["ms_per_fine_step_periodic_x"] = bench_open_dune(hl, wl, stream, open_faces=False)["ms_per_fine_step"]
        else:
            pos0 = torch.tensor(wl.particle_cloud(512), device="cuda")
            bench_multilevel(hl, wl, stream, "f32", pos0, fine_steps=48)
            res = bench_multilevel(hl, wl, stream, "f32", pos0, profile=args.profile)[0]
        print(json.dumps({"only": args.only, "result": res}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    config = {"workload": "duct %d^3, periodic x, bounce-back y/z, 8^3 blocks, tau 0.55, F=1e-6" % args.n,
              "nodes": args.n ** 3, "storage": args.storage, "l2": "inputs (2 x %.0f MB) larger than the 129 MB L2"
              % (args.n ** 3 * STORAGE_BYTES[args.storage] / 2 / 1e6), "parallelism": "replicas x%d" % world}

    if args.impl == "reference":
        if rank != 0:
            return
        steps = max(1, min(args.steps, 8))
        cb = cpu_oracle_sample(128, steps)
        cb["nproc"] = os.cpu_count()
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS",
                          "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": config, "cpu_baseline": cb,
                          "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_gpu(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    bpn = STORAGE_BYTES[args.storage]
    achieved = args.n ** 3 * bpn / (res["ms_per_step"] / 1e3) / 1e9
    # DRAM bytes per node update from the ncu captures of the 192^3 duct (the
    # FP32 and FP16 kernels; none taken for BF16)
    traffic = {"f32": TRAFFIC_PER_NODE, "f16s": (147.631104e6 + 106.398720e6) / 192 ** 3}.get(args.storage)
    line = {
        "metric": METRIC,
        "value": round(res["value"], 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(res["ms_per_step"], 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.storage,
        "data": "synthetic",
        "config": config,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": None if traffic is None else round(traffic * args.n ** 3),
                     "kernel": STORAGE_KERNEL[args.storage], "peak_kind": peak_kind,
                     "bytes_per_node": bpn},
        "e2e": {"value": round(res["e2e_value"], 1), "unit": "MLUPS",
                "h2d_bytes_per_step": int(res["e2e_bytes"] // args.steps),
                "d2h_bytes_per_step": int((res["e2e_bytes"] + 56) // args.steps)},
        "gpu_launches": args.steps,
        "clocks": res["clocks"],
    }
    if res["extras"] is not None:
        line["extras"] = res["extras"]
        if FLOP_PER_NODE is not None:
            # the same kernel against the FP32 CUDA-core rate (the kernel is issue-bound, not HBM-bound)
            tf = args.n ** 3 * FLOP_PER_NODE / (res["ms_per_step"] / 1e3) / 1e12
            pk = res["extras"].get("fp32_sgemm_tflops")
            line["extras"]["alu_roofline"] = {
                "kernel": STORAGE_KERNEL[args.storage], "flop_per_node": FLOP_PER_NODE, "achieved_tflops": round(tf, 2),
                "peak_tflops": pk, "peak_kind": "cuBLAS SGEMM 8192^3, TF32 off, measured in this run",
                "frac": round(tf / pk, 4) if pk else None}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    ex = res["extras"]
    if ex is not None:
        # compact figures of the secondary workloads, last on the line
        c5 = ex["c5_batched"]["f16s"]
        c3 = ex["c3_multilevel"]
        line["summary"] = {
            "duct_f32_frac": line["roofline"]["frac"],
            "duct_f16s_mlups": ex["duct_f16s"]["mlups"], "duct_f16s_frac": ex["duct_f16s"]["frac"],
            "duct_f16s_over_f32": round(ex["duct_f16s"]["mlups"] / line["value"], 3),
            "c5_mlups": c5["mlups"], "c5_frac": round(c5["hbm_gbs"] / peak, 4), "c5_mode": c5["mode"],
            "c4_adjoint_over_forward": ex["c4_adjoint"]["adjoint_over_forward"],
            "c3_f32_mlups": c3["f32"]["mlups_fine_equiv"],
            "c3_actual_gbs_over_peak": c3["f32"]["actual_gbs_over_peak"],
            "c3_f16s_over_f32": round(c3["f16s"]["mlups_fine_equiv"] / c3["f32"]["mlups_fine_equiv"], 3),
            "c3_rebuild_share": round(c3["f32"]["rebuild_s"] / c3["f32"]["total_s"], 4),
            "c3_adjoint_over_forward": ex["c3_adjoint"]["adjoint_over_forward"],
            "sparse_2048_mlups": ex["sparse_tree_2048"]["mlups_fine_equiv"],
            "open_dune_mlups": ex["f3_open_dune"]["mlups_fine_equiv"],
            "open_dune_over_periodic": round(ex["f3_open_dune"]["ms_per_fine_step_periodic_x"] /
                                             ex["f3_open_dune"]["ms_per_fine_step"], 3),
        }
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
