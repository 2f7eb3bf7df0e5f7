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
not shard in this build): value = all ranks' node updates / the slowest rank.
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
TRAFFIC_PER_NODE = 532.3e6 / 192 ** 3


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


def duct_lattice(hl, n, stream):
    lat = hl.Lattice((n, n, n), tau=0.55, periodic=(True, False, False), storage="f32", stream=stream)
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
    lat = duct_lattice(hl, n, stream.cuda_stream)
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
    lat = duct_lattice(hl, n, stream.cuda_stream)
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
    times = torch.tensor([ms / 1e3, t_e2e], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(times, op=torch.distributed.ReduceOp.MAX)
    t_dev, t_e2e = times.tolist()
    res = {
        "ms_per_step": 1e3 * t_dev / args.steps,
        "value": world * nodes * args.steps / t_dev / 1e6,
        "e2e_value": world * nodes * args.steps / t_e2e / 1e6,
        "clocks": clk,
        "mass": red[0],
        "e2e_bytes": M0.nbytes,
        "finite": bool(np.isfinite(red_e2e[0])),
    }
    return res


def cpu_oracle_sample(n_sample=64, steps=12):
    """The FP64 CPU oracle on an n_sample^3 duct of the same kind (bounded sample)."""
    import torch
    from oracle import single_level as sl
    from paper_2603_14982_gb300 import workloads as wl

    M = torch.tensor(wl.rest_field((n_sample,) * 3))
    blocked = sl.blocked_sources(M.shape[1:], (True, False, False))
    sl.step(M, 0.55, force=(1e-6, 0, 0), periodic=(True, False, False), blocked=blocked)
    t0 = time.perf_counter()
    for _ in range(steps):
        M = sl.step(M, 0.55, force=(1e-6, 0, 0), periodic=(True, False, False), blocked=blocked)
    dt = time.perf_counter() - t0
    return {"value": n_sample ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": torch.get_num_threads(),
            "kind": "oracle", "sample": "%d^3 duct of the same kind, %d steps, FP64 torch CPU, %.1f s" %
            (n_sample, steps, dt)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    config = {"workload": "duct %d^3, periodic x, bounce-back y/z, 8^3 blocks, tau 0.55, F=1e-6" % args.n,
              "nodes": args.n ** 3, "storage": "f32", "l2": "inputs (2 x %.0f MB) larger than the 129 MB L2"
              % (args.n ** 3 * 40 / 1e6), "parallelism": "replicas x%d" % world}

    if args.impl == "reference":
        if rank != 0:
            return
        steps = max(1, min(args.steps, 8))
        cb = cpu_oracle_sample(128, steps)
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
    achieved = args.n ** 3 * BYTES_PER_NODE_F32 / (res["ms_per_step"] / 1e3) / 1e9
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
        "dtype": "f32",
        "data": "synthetic",
        "config": config,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": None if TRAFFIC_PER_NODE is None else round(TRAFFIC_PER_NODE * args.n ** 3),
                     "kernel": KERNEL, "peak_kind": peak_kind,
                     "bytes_per_node": BYTES_PER_NODE_F32},
        "e2e": {"value": round(res["e2e_value"], 1), "unit": "MLUPS",
                "h2d_bytes_per_step": int(res["e2e_bytes"] // args.steps),
                "d2h_bytes_per_step": int((res["e2e_bytes"] + 56) // args.steps)},
        "gpu_launches": args.steps,
        "clocks": res["clocks"],
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_oracle_sample(128, 16)
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
