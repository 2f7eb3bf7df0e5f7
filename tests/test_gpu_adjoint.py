"""GPU adjoint (hlbm_forward_record / hlbm_adjoint behind torch.autograd) vs references.

Loss (obstacle channel): L = 1/2 sum over the last x-plane of rho |u|^2 with the
physical velocity u = u' - F/(2 rho), as a function of the per-node force F.
* small channel: the GPU gradient (FP32 and FP64 storage) against the oracle's
  FP64 reverse-mode gradient, relative to max |dL/dF|: 1e-4 (FP32 storage),
  1e-6 (FP64 storage: the adjoint variables and dL/dF are float32);
* the 128^3 channel with the 16^3 obstacle, 200 steps, checkpoints every 20:
  the FP32 adjoint against central differences of the FP64 GPU forward on 32
  random fluid cells of the whole channel, within 1e-4 of max |dL/dF|.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def outlet_mask(lat, nx):
    coords, _ = lat.blocks(0)
    x = coords[:, 0:1] * 8 + (np.arange(512)[None, :] & 7)
    return torch.tensor(x == nx - 1, device="cuda")


def loss_fn(M, F, mask):
    """L from block-layout stored moments M [n][10][512] and force F [n][3][512] (float64 math)."""
    M = M.double()
    F = F.double()
    rho = M[:, 0]
    u = [M[:, 1 + a] - 0.5 * F[:, a] / rho for a in range(3)]
    ke = 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    return (ke * mask).sum()


def gpu_gradient(M0, F, solid, extent, steps, ckpt, tau, storage, periodic):
    nx, ny, nz = extent
    with hl.Lattice(extent, tau=tau, periodic=periodic, storage=storage) as lat:
        lat.set_dense()
        if solid is not None:
            lat.set_solid(solid)
        lat.write_moments(hl.dense_to_blocks(M0))
        Fb = torch.tensor(hl.dense_to_blocks(F), dtype=torch.float32, device="cuda").requires_grad_(True)
        fwd = hl.make_force_autograd(lat, steps, ckpt)
        M = fwd(Fb)
        L = loss_fn(M, Fb, outlet_mask(lat, nx))
        L.backward()
        g = Fb.grad.detach().double().cpu().numpy()
    return L.item(), hl.blocks_to_dense(g, (nz, ny, nx))


def small_case():
    extent = (32, 16, 16)
    nx, ny, nz = extent
    shape = (nz, ny, nx)
    solid = np.zeros(shape, dtype=np.uint8)
    solid[6:10, 6:10, 12:16] = 1
    M0 = wl.random_field(shape, 91, du=0.02, drho=1e-3, dneq=1e-4)
    M0[:, solid.astype(bool)] = wl.rest_field((1, 1, 1))[:, 0, 0, :1]
    F = wl.noisy_force(shape, seed=92, mean=(1e-5, 0.0, 0.0), sigma=1e-5)
    return extent, shape, solid, M0, F


@pytest.mark.parametrize("storage,tol", [("f32", 1e-4), ("f64", 1e-6)])
def test_gradient_matches_oracle_reverse_mode(storage, tol):
    extent, shape, solid, M0, F = small_case()
    per = (True, False, False)
    # the oracle starts from the state the GPU stores and the force it uses
    with hl.Lattice(extent, tau=0.7, periodic=per, storage=storage) as lat:
        lat.set_dense()
        lat.write_moments(hl.dense_to_blocks(M0))
        start = hl.blocks_to_dense(lat.read_moments(), shape)
    Fq = F.astype(np.float32).astype(np.float64)
    Lg, g = gpu_gradient(start, Fq, solid, extent, 12, 5, 0.7, storage, per)
    Lo, go = oadj.gradient(torch.tensor(start), torch.tensor(Fq), 12, 0.7, per, solid=torch.tensor(solid.astype(bool)))
    go = go.numpy()
    assert abs(Lg - Lo.item()) <= 1e-5 * abs(Lo.item())
    fluid = ~solid.astype(bool)
    err = np.abs(g - go)[:, fluid].max() / np.abs(go).max()
    print("%s adjoint, 12 steps with an obstacle: max |g - oracle| / max |g| = %.2e" % (storage, err))
    assert err < tol, err


def test_obstacle_channel_128_central_differences():
    n, steps, ckpt = 128, 200, 20
    extent = (n, n, n)
    shape = (n, n, n)
    solid = wl.obstacle_mask(n).astype(np.uint8)
    F = wl.noisy_force(shape).astype(np.float32)
    M0 = wl.rest_field(shape)
    per = (True, False, False)
    L, g = gpu_gradient(M0, F.astype(np.float64), solid, extent, steps, ckpt, 0.55, "f32", per)
    # central differences with the FP64 forward on 32 random fluid cells of
    # the whole channel, one random force component each
    rng = np.random.default_rng(5)
    cells = []
    while len(cells) < 32:
        z, y, x = (int(v) for v in rng.integers(0, n, 3))
        if not solid[z, y, x]:
            cells.append((z, y, x, int(rng.integers(0, 3))))
    with hl.Lattice(extent, tau=0.55, periodic=per, storage="f64") as lat:
        lat.set_dense()
        lat.set_solid(solid)
        mask = outlet_mask(lat, n)
        M0b = torch.tensor(hl.dense_to_blocks(M0), device="cuda")
        Fb0 = torch.tensor(hl.dense_to_blocks(F), device="cuda")

        def L_of(Fb):
            lat.write_moments(M0b)
            lat.set_force(Fb)
            lat.step(steps)
            M = torch.empty((lat.num_blocks(0), 10, 512), dtype=torch.float64, device="cuda")
            lat.read_moments(M)
            return loss_fn(M, Fb, mask).item()

        coords, _ = lat.blocks(0)
        index = {tuple(c): i for i, c in enumerate(coords.tolist())}
        gmax = np.abs(g).max()
        worst = 0.0
        for (z, y, x, a) in cells:
            b = index[(x // 8, y // 8, z // 8)]
            c = (x % 8) + 8 * (y % 8) + 64 * (z % 8)
            h = 1e-3 * abs(float(F[a, z, y, x])) + 1e-9
            Fp = Fb0.clone()
            Fp[b, a, c] += h
            Fm = Fb0.clone()
            Fm[b, a, c] -= h
            hp = float(Fp[b, a, c] - Fb0[b, a, c])   # the float32 step actually taken
            hm = float(Fb0[b, a, c] - Fm[b, a, c])
            fd = (L_of(Fp) - L_of(Fm)) / (hp + hm)
            worst = max(worst, abs(g[a, z, y, x] - fd) / gmax)
            assert abs(g[a, z, y, x] - fd) <= 1e-4 * gmax, (z, y, x, a, g[a, z, y, x], fd, gmax)
    print("C4 central differences: 32 cells, max |g - fd| / max |g| = %.2e" % worst)
