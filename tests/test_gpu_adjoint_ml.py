"""Adjoint of the multi-level advance on the GPU (FP32 storage) against the
oracle's FP64 reverse mode and against central finite differences.

* two levels (periodic band) and three levels (a patch on a wall): dL/dF of
  L = sum_l <W_l, M_l> through sub-cycling, both transfers with their S^neq
  rescaling, interface copy nodes and bounce-back, with checkpoint segments
  of one and two coarse steps; within 1e-4 of the largest gradient entry;
* the same gradient against central differences of the GPU's own FP64-storage
  forward run at single cells, on the small cases and on the full-size
  512^3 hierarchy of the 2M-particle cloud;
* the torch.autograd.Function over all levels gives the same gradient;
* a rebuild between the recorded run and the adjoint is refused, and so is
  reduced-precision storage.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as adj
from paper_2603_14982_gb300 import homelbm as hl
from tests.helpers import ml_adjoint_case

pytestmark = pytest.mark.gpu


def gpu_lattice(c, storage="f32"):
    lat = hl.Lattice(c["ext"], levels=c["L"], tau=c["tau0"], periodic=c["periodic"], storage=storage)
    z, y, x = np.nonzero(c["O0"])
    lat.set_fine_blocks(np.stack([x, y, z], axis=1))
    coords = []
    for l in range(c["L"]):
        cl, _ = lat.blocks(l)
        assert np.array_equal(cl, c["h"].blocks(l))
        coords.append(cl)
        lat.write_moments(hl.dense_to_blocks(c["M0"][l], cl), level=l)
    return lat, coords


def start_state(lat, c, coords):
    """The GPU's stored start state as dense FP64 fields (what the oracle starts from)."""
    out = []
    for l in range(c["L"]):
        shape = c["h"].stored_nodes(l).shape
        out.append(hl.blocks_to_dense(lat.read_moments(level=l), shape, coords[l], fill=0.0))
    return out


def run_adjoint(lat, c, coords, F32, W32):
    Fb = torch.tensor(hl.dense_to_blocks(F32, coords[0]), device="cuda")
    lat.set_force(Fb)
    per = 1 << (c["L"] - 1)
    lat.forward_record(c["n_coarse"] * per, c["ckpt"] * per)
    dLdM = torch.cat([torch.tensor(hl.dense_to_blocks(W32[l], coords[l]), device="cuda")
                      for l in range(c["L"])])
    dF = torch.empty((len(coords[0]), 3, 512), dtype=torch.float32, device="cuda")
    lat.adjoint(dLdM, dF)
    return dF.cpu().numpy()


@pytest.mark.parametrize("name", ["two_level", "three_level_wall"])
def test_ml_adjoint_matches_oracle_reverse_mode(name):
    c = ml_adjoint_case(name)
    F32 = c["F"].astype(np.float32)
    W32 = [w.astype(np.float32) for w in c["W"]]
    lat, coords = gpu_lattice(c)
    with lat:
        M0 = start_state(lat, c, coords)
        got = run_adjoint(lat, c, coords, F32, W32)
    _, g = adj.ml_gradient(c["h"], c["tau0"], M0, F32.astype(np.float64), c["n_coarse"],
                           [w.astype(np.float64) for w in W32])
    ref = hl.dense_to_blocks(g.numpy(), coords[0])
    scale = np.abs(ref).max()
    assert scale > 0
    err = np.abs(got - ref).max() / scale
    print("%s multi-level adjoint: max |g - oracle| / max |g| = %.2e" % (name, err))
    assert err < 1e-4, err


def test_ml_adjoint_matches_central_differences():
    c = ml_adjoint_case("two_level")
    F32 = c["F"].astype(np.float32)
    W32 = [w.astype(np.float32) for w in c["W"]]
    lat, coords = gpu_lattice(c)
    with lat:
        got = run_adjoint(lat, c, coords, F32, W32)
    per = 1 << (c["L"] - 1)
    Wb = [hl.dense_to_blocks(W32[l].astype(np.float64), coords[l]) for l in range(c["L"])]

    def loss(F):
        lat, cs = gpu_lattice(c, storage="f64")
        with lat:
            lat.set_force(torch.tensor(hl.dense_to_blocks(F, cs[0]).astype(np.float32), device="cuda"))
            lat.step(c["n_coarse"] * per)
            return sum(float((lat.read_moments(level=l) * Wb[l]).sum()) for l in range(c["L"]))

    rng = np.random.default_rng(23)
    h = 2.0 ** -17  # exact in FP32 next to |F| ~ 1e-5
    scale = np.abs(got).max()
    worst = 0.0
    for _ in range(4):
        b, r, n = int(rng.integers(len(coords[0]))), int(rng.integers(3)), int(rng.integers(512))
        x = coords[0][b, 0] * 8 + n % 8
        y = coords[0][b, 1] * 8 + (n // 8) % 8
        z = coords[0][b, 2] * 8 + n // 64
        Fp, Fm = F32.copy(), F32.copy()
        Fp[r, z, y, x] += h
        Fm[r, z, y, x] -= h
        fd = (loss(Fp) - loss(Fm)) / (float(np.float32(F32[r, z, y, x] + h)) - float(np.float32(F32[r, z, y, x] - h)))
        assert abs(fd - got[b, r, n]) < 1e-4 * scale, (b, r, n, fd, got[b, r, n])
        worst = max(worst, abs(fd - got[b, r, n]) / scale)
    print("multi-level adjoint, central differences on 4 cells: max |g - fd| / max |g| = %.2e" % worst)


def test_ml_autograd_function_and_refusals():
    c = ml_adjoint_case("two_level")
    F32 = c["F"].astype(np.float32)
    W32 = [w.astype(np.float32) for w in c["W"]]
    lat, coords = gpu_lattice(c)
    per = 1 << (c["L"] - 1)
    with lat:
        direct = run_adjoint(lat, c, coords, F32, W32)
        # back to the start state for the autograd run
        for l in range(c["L"]):
            lat.write_moments(hl.dense_to_blocks(c["M0"][l], coords[l]), level=l)
        f = hl.make_force_autograd(lat, c["n_coarse"] * per, c["ckpt"] * per)
        F = torch.tensor(hl.dense_to_blocks(F32, coords[0]), device="cuda", requires_grad=True)
        out = f(F)
        assert out.shape[0] == sum(len(x) for x in coords)
        W = torch.cat([torch.tensor(hl.dense_to_blocks(W32[l], coords[l]), device="cuda") for l in range(c["L"])])
        (out * W).sum().backward()
        # equal up to the order of the FP32 atomic sums of the transposed downward transfer
        assert np.abs(F.grad.cpu().numpy() - direct).max() <= 1e-6 * np.abs(direct).max()
        # a rebuild changes the block layout: the recorded run no longer applies
        z, y, x = np.nonzero(c["O0"])
        lat.set_fine_blocks(np.stack([x, y, z], axis=1))
        dF = torch.empty_like(F)
        with pytest.raises(hl.HlbmError) as ei:
            lat.adjoint(W, dF)
        assert ei.value.code == hl.E_BAD_STATE
    lat, coords = gpu_lattice(c, storage="f16s")
    with lat:
        with pytest.raises(hl.HlbmError) as ei:
            lat.forward_record(2 * per, per)
        assert ei.value.code == hl.E_UNSUPPORTED


def test_ml_adjoint_full_size_cloud_central_differences():
    """The 512^3 three-level hierarchy of the 2M-particle cloud (the one the
    multi-level benchmarks use), 8 fine steps from rest under a seeded force
    field, checkpoints every 4: dL/dF of L = sum_l <W_l, M_l> (W seeded on
    every stored node) from the FP32 adjoint against central differences of
    the GPU's FP64-storage forward run at 4 level-0 entries (the largest, and
    three drawn among those above 1 % of it), within 1e-4 of max |dL/dF| as
    on the small cases."""
    from paper_2603_14982_gb300 import workloads as wl
    n, L, steps, ckpt = 512, 3, 8, 4
    ext, per = (n, n, n), (True, False, True)
    pos = torch.tensor(wl.particle_cloud(n), device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(29)
    with hl.Lattice(ext, levels=L, tau=0.9, periodic=per, storage="f32") as lat:
        lat.rebuild_from_particles(pos)
        counts = [lat.num_blocks(l) for l in range(L)]
        F = 1e-5 * torch.randn((counts[0], 3, 512), generator=gen, device="cuda", dtype=torch.float32)
        W = [torch.randn((c, 10, 512), generator=gen, device="cuda", dtype=torch.float32) for c in counts]
        lat.set_force(F)
        lat.forward_record(steps, ckpt)
        g = torch.empty((counts[0], 3, 512), dtype=torch.float32, device="cuda")
        lat.adjoint(torch.cat(W), g)
    g = g.double()
    scale = float(g.abs().max())
    assert scale > 0 and torch.isfinite(g).all()

    def loss(Fp):
        with hl.Lattice(ext, levels=L, tau=0.9, periodic=per, storage="f64") as lat:
            lat.rebuild_from_particles(pos)
            assert [lat.num_blocks(l) for l in range(L)] == counts
            lat.set_force(Fp)
            lat.step(steps)
            total = 0.0
            for l in range(L):
                M = torch.empty((counts[l], 10, 512), dtype=torch.float64, device="cuda")
                lat.read_moments(M, level=l)
                total += float((M * W[l].double()).sum())
            return total

    # the largest entry and three random entries above 1 % of it
    flat = g.abs().flatten()
    big = torch.nonzero(flat > 0.01 * scale).flatten().cpu().numpy()
    rng = np.random.default_rng(31)
    picks = [int(torch.argmax(flat))] + [int(v) for v in rng.choice(big, 3, replace=False)]
    h = 2.0 ** -17
    worst = 0.0
    for k in picks:
        b, r, c = k // (3 * 512), (k // 512) % 3, k % 512
        Fp, Fm = F.clone(), F.clone()
        Fp[b, r, c] += h
        Fm[b, r, c] -= h
        fd = (loss(Fp) - loss(Fm)) / (float(Fp[b, r, c]) - float(Fm[b, r, c]))
        worst = max(worst, abs(fd - float(g[b, r, c])) / scale)
        assert abs(fd - float(g[b, r, c])) < 1e-4 * scale, (b, r, c, fd, float(g[b, r, c]), scale)
    print("512^3 cloud hierarchy, multi-level adjoint against central differences: max |g - fd| / max |g| = %.2e"
          % worst)
