"""Shared test helpers: error metrics and single-node oracle updates."""
import numpy as np
import torch

from oracle import single_level as sl

# Per-row floors of the error scale: rho ~ 1, u ~ U, S ~ U^2.
def row_scales(ref, u_floor=1e-3):
    """max |ref| per moment row, floored (rho: 1, u: u_floor, S: u_floor^2)."""
    R = ref.shape[0]
    flat = np.abs(ref.reshape(R, -1))
    flat = np.where(np.isfinite(flat), flat, 0.0)
    s = flat.max(axis=1)
    floor = np.array([1.0] + [u_floor] * 3 + [u_floor ** 2] * 6)[:R]
    return np.maximum(s, floor)


def rel_err(got, ref, scales=None, mask=None):
    """max over nodes of |got - ref| / scale_row, per row (array of 10)."""
    if scales is None:
        scales = row_scales(ref)
    d = np.abs(np.asarray(got, dtype=np.float64) - np.asarray(ref, dtype=np.float64))
    R = d.shape[0]
    d = d.reshape(R, -1)
    if mask is not None:
        d = d[:, np.asarray(mask).reshape(-1)]
    return d.max(axis=1) / scales


def oracle_node_update(M, nodes, tau, periodic, force=None, eps=None, solid=None, mode="hermite"):
    """Oracle step of single nodes of a large dense field, one 3^3 patch at a time.

    M: (10, nz, ny, nx) float64; nodes: list of (x, y, z).  The patch is taken
    with periodic wrap; pulls that cross a wall or hit a solid node are marked
    blocked exactly as on the full grid.  Returns (10, n) float64.
    """
    nz, ny, nx = M.shape[1:]
    ext = (nx, ny, nz)
    out = []
    for (x, y, z) in nodes:
        idx = [np.arange(c - 1, c + 2) for c in (z, y, x)]
        zi, yi, xi = (i % n for i, n in zip(idx, (nz, ny, nx)))
        P = torch.tensor(M[:, zi][:, :, yi][:, :, :, xi])
        blocked = []
        for c in sl.lat.C:
            b = torch.zeros((3, 3, 3), dtype=torch.bool)
            src = (x - c[0], y - c[1], z - c[2])
            hit = any((not periodic[a]) and not (0 <= src[a] < ext[a]) for a in range(3))
            if solid is not None and not hit:
                hit = bool(solid[src[2] % nz, src[1] % ny, src[0] % nx])
            b[1, 1, 1] = hit
            blocked.append(b)
        Fp = None
        if force is not None:
            Fp = force if isinstance(force, tuple) else torch.tensor(force[:, zi][:, :, yi][:, :, :, xi])
        ep = None if eps is None else torch.tensor(eps[zi][:, yi][:, :, xi])
        sp = None if solid is None else torch.tensor(solid[zi][:, yi][:, :, xi].astype(bool))
        Mn = sl.step(P, tau, force=Fp, eps=ep, periodic=(True, True, True), solid=sp, mode=mode, blocked=blocked)
        out.append(Mn[:, 1, 1, 1].numpy())
    return np.stack(out, axis=1)


# Multi-level adjoint cases: a hierarchy, per-level dense initial fields (a
# shear wave), a seeded level-0 force field and loss weights W_l (zero where
# level l stores no node) for L = sum_l <W_l, M_l> after n_coarse coarse steps.
ML_ADJOINT_CASES = {
    # two levels, fully periodic: a refined band across the domain
    "two_level": dict(ext=(16, 128, 16), L=2, band=(slice(None), slice(7, 9), slice(None)),
                      periodic=(True, True, True), tau0=0.8, n_coarse=3, ckpt=2),
    # three levels, a refined patch on the floor wall (bounce-back at y = 0, 127)
    "three_level_wall": dict(ext=(32, 128, 32), L=3, band=(slice(1, 3), slice(0, 2), slice(1, 3)),
                             periodic=(True, False, True), tau0=0.9, n_coarse=2, ckpt=1),
}


def ml_adjoint_case(name, seed=11):
    from oracle import hierarchy as hy
    from oracle import multilevel as ml
    from paper_2603_14982_gb300 import workloads as wl
    c = dict(ML_ADJOINT_CASES[name])
    ext, L = c["ext"], c["L"]
    O0 = np.zeros(hy.block_dims(ext, 8, 0), bool)
    O0[c["band"]] = True
    h = hy.Hierarchy(O0, ext, 8, L, c["periodic"])
    m = ml.MultiLevel(h, c["tau0"])
    M0 = []
    for l in range(L):
        X, Y, Z = m.node_positions(l)
        ux = 0.01 * np.sin(2 * np.pi * Y / ext[1])
        M0.append(wl.equilibrium_field(np.ones_like(ux) + 1e-3 * np.cos(2 * np.pi * X / 16), ux, 0.3 * ux,
                                       np.zeros_like(ux)))
    rng = np.random.default_rng(seed)
    F = rng.normal(0.0, 1e-5, (3,) + m.shape[0])
    W = [rng.normal(size=(10,) + m.shape[l]) * m.stored[l].numpy() for l in range(L)]
    c.update(O0=O0, h=h, M0=M0, F=F, W=W, stored=[m.stored[l].numpy() for l in range(L)])
    return c
