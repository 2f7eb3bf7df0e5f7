"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds no arithmetic of the method itself: it only draws initial
moment fields, particle clouds, force/solid-fraction fields and obstacle masks.
Everything is numpy float64 on the host (callers cast and copy).  Field arrays
are indexed [z, y, x]; a moment field is (10, nz, ny, nx) with rows
(rho, u_x, u_y, u_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz).

The workload shapes follow the paper's use: a Taylor-Green vortex and a
force-driven duct for the single-level path, a falling particle cloud that
drives refinement (the paper's MPM particles enter only through the level
selection Phi and the force/solid-fraction fields, Sec. 5.4), an obstacle
channel for the gradient, a batch of uneven periodic domains, and a
branching tube tree that refines a 2048^3 domain sparsely (the paper's airway
scene, where refinement follows the tube walls, Sec. 7 and Table 1).
"""
import numpy as np

# Seeds per workload.
SEED_TGV, SEED_DUCT, SEED_CLOUD, SEED_ADJOINT, SEED_BATCH, SEED_TREE = 1, 2, 3, 4, 5, 17


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _pack(rho, ux, uy, uz, sxx, syy, szz, sxy, sxz, syz):
    return np.stack([rho, ux, uy, uz, sxx, syy, szz, sxy, sxz, syz]).astype(np.float64)


def equilibrium_field(rho, ux, uy, uz):
    """A moment field whose second-order moment is the equilibrium one, S = u u."""
    return _pack(rho, ux, uy, uz, ux * ux, uy * uy, uz * uz, ux * uy, ux * uz, uy * uz)


def taylor_green_3d(n, u0=0.05):
    """3D Taylor-Green vortex on an n^3 periodic box, k = 2 pi / n.

    u = U0 sin kx cos ky cos kz, v = -U0 cos kx sin ky cos kz, w = 0, with the
    matching pressure rho = 1 + 3 U0^2/16 (cos 2kx + cos 2ky)(cos 2kz + 2).
    """
    k = 2.0 * np.pi / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ux = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    uy = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    uz = np.zeros_like(ux)
    rho = 1.0 + 3.0 * u0 * u0 / 16.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (np.cos(2 * k * z) + 2.0)
    return equilibrium_field(rho, ux, uy, uz)


def taylor_green_2d(n, nz=1, u0=0.05):
    """z-invariant Taylor-Green vortex (an exact Navier-Stokes solution)."""
    k = 2.0 * np.pi / n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    ux = u0 * np.sin(k * x) * np.cos(k * y)
    uy = -u0 * np.cos(k * x) * np.sin(k * y)
    uz = np.zeros_like(ux)
    rho = 1.0 - 3.0 * u0 * u0 / 4.0 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    return equilibrium_field(rho, ux, uy, uz)


def rest_field(shape):
    """rho = 1, u = 0, S = 0 on a (nz, ny, nx) grid."""
    z = np.zeros(shape)
    return _pack(np.ones(shape), z, z, z, z, z, z, z, z, z)


def random_field(shape, seed, du=0.02, drho=0.01, dneq=2e-3):
    """Smooth-free random moments: rho = 1 + drho*N, u = du*N, S = u u + dneq*N."""
    g = rng(seed)
    rho = 1.0 + drho * g.standard_normal(shape)
    ux, uy, uz = (du * g.standard_normal(shape) for _ in range(3))
    m = equilibrium_field(rho, ux, uy, uz)
    m[4:] += dneq * g.standard_normal((6,) + tuple(shape))
    return m


def shear_wave(shape, amp=0.01, axis_flow=0, axis_var=1, periods=1):
    """u_{flow} = amp sin(2 pi periods y / n_y) along axis_var, S = u u."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coord = (x, y, z)[axis_var]
    n = (nx, ny, nz)[axis_var]
    u = [np.zeros(shape) for _ in range(3)]
    u[axis_flow] = amp * np.sin(2 * np.pi * periods * coord / n)
    return equilibrium_field(np.ones(shape), u[0], u[1], u[2])


# --- particle cloud that drives refinement (stand-in for the MPM particles) ---

def particle_cloud(n_fine, count=2_000_000, seed=SEED_CLOUD, box=(0.2, 0.4, 0.2), y0_frac=0.05):
    """Jittered-lattice cloud in a box of the given domain fractions.

    The box spans box*n_fine cells, centred in x and z; its bottom sits at
    y0_frac*n_fine.  ``count`` particles on an (a, 2a, a) lattice (a^3*2 =
    count), each jittered uniformly by +-1/2 lattice spacing.  Returns float32
    positions (count, 3) in fine-cell units (x, y, z).
    """
    g = rng(seed)
    a = int(round((count / 2) ** (1.0 / 3.0)))
    dims = (a, 2 * a, a)
    ext = np.array(box) * n_fine
    lo = np.array([(n_fine - ext[0]) / 2.0, y0_frac * n_fine, (n_fine - ext[2]) / 2.0])
    sp = ext / np.array(dims)
    iz, iy, ix = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    idx = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = lo + (idx + 0.5 + g.uniform(-0.5, 0.5, idx.shape)) * sp
    return pos.astype(np.float32)


def sand_heap(extent, count=600_000, seed=SEED_CLOUD, x0_frac=0.4, sigma_frac=0.12, height_frac=0.25):
    """Particles (float32 (count, 3), fine-node units) filling a dune-shaped heap
    on the floor y = 0 of an extent = (nx, ny, nz) domain: the heap spans z,
    its height along x is height_frac ny exp(-((x - x0) / sigma)^2 / 2) with
    x0 = x0_frac nx and sigma = sigma_frac nx; particles are drawn uniformly
    under that profile (seeded)."""
    nx, ny, nz = extent
    g = np.random.default_rng(seed)
    x0, sig, top = x0_frac * nx, sigma_frac * nx, height_frac * ny
    out = np.empty((0, 3))
    while len(out) < count:  # rejection sampling of the area under the profile
        m = 2 * (count - len(out)) + 1024
        x = g.uniform(0.0, nx, m)
        y = g.uniform(0.0, top, m)
        keep = y < top * np.exp(-0.5 * ((x - x0) / sig) ** 2)
        z = g.uniform(0.0, nz, m)
        out = np.concatenate([out, np.stack([x, y + 0.5, z], axis=1)[keep]])
    return out[:count].astype(np.float32)


def fall(pos, steps, floor=0.5):
    """Move the cloud down by one cell per step, clamped at the floor."""
    out = pos.copy()
    out[:, 1] = np.maximum(out[:, 1] - float(steps), floor)
    return out


# --- gradient workload: channel with a central obstacle ---

def obstacle_mask(n, lo=None, hi=None):
    """Bool (n, n, n) mask of the solid cube [lo, hi)^3 (default: centred, n/8 wide)."""
    if lo is None:
        lo = n // 2 - n // 16
        hi = n // 2 + n // 16
    m = np.zeros((n, n, n), dtype=bool)
    m[lo:hi, lo:hi, lo:hi] = True
    return m


def noisy_force(shape, seed=SEED_ADJOINT, mean=(1e-6, 0.0, 0.0), sigma=1e-6):
    """F(x) = mean + sigma * N(0, 1) per component per cell, float64 (3, nz, ny, nx)."""
    g = rng(seed)
    F = sigma * g.standard_normal((3,) + tuple(shape))
    for a in range(3):
        F[a] += mean[a]
    return F


# --- batch of uneven periodic domains ---

def batch_domains(count=64, seed=SEED_BATCH, edges=(32, 48, 64, 96, 128),
                  amp=(0.01, 0.08), tau=(0.52, 0.8)):
    """List of (edge, U0, tau) for independent periodic Taylor-Green domains."""
    g = rng(seed)
    out = []
    for _ in range(count):
        e = int(g.choice(edges))
        out.append((e, float(g.uniform(*amp)), float(g.uniform(*tau))))
    return out


# --- sparse domain: a branching tube tree ---

def tube_tree_blocks(n_fine=2048, generations=9, seed=SEED_TREE, r0_frac=0.025, l0_frac=0.2,
                     shrink_r=2.0 ** (-1.0 / 3.0), shrink_l=0.72, angle=0.6, block=8):
    """Level-0 blocks (int32 (n, 3) as (bx, by, bz), sorted by slot id) that a
    seeded binary tube tree's walls pass through.

    The trunk starts near the top of the domain (y = 0.95 n) and points down
    (-y).  Each tube splits into two whose directions turn by about ``angle``
    rad to either side within a plane that rotates with every generation;
    radii shrink by 2^(-1/3) per generation and lengths by ``shrink_l`` (with
    10-15 % seeded jitter on angles and lengths).  The walls are sampled about
    every two fine nodes.  With the defaults and four levels the hierarchy
    stores about 40 times fewer nodes than the 2048^3 domain, the sparsity of
    the paper's airway scene (41.4x).
    """
    g = rng(seed)
    n = float(n_fine)
    nb = n_fine // block
    occ = np.zeros((nb, nb, nb), dtype=bool)
    stack = [(np.array([n / 2, 0.95 * n, n / 2]), np.array([0.0, -1.0, 0.0]), np.array([1.0, 0.0, 0.0]),
              r0_frac * n, l0_frac * n, 0)]
    segments = []
    while stack:
        p, d, side, r, length, gen = stack.pop()
        q = p + d * length
        segments.append((p, q, r))
        if gen + 1 >= generations:
            continue
        for s in (-1.0, 1.0):
            a = angle * (1.0 + 0.15 * g.standard_normal())
            nd = np.cos(a) * d + s * np.sin(a) * side
            nd /= np.linalg.norm(nd)
            ns = np.cross(nd, side)
            ns /= np.linalg.norm(ns)
            stack.append((q, nd, ns, r * shrink_r, length * shrink_l * (1.0 + 0.1 * g.standard_normal()), gen + 1))
    for p, q, r in segments:
        d = q - p
        length = np.linalg.norm(d)
        d = d / length
        u = np.cross(d, [0.3, 0.5, 0.8])
        u /= np.linalg.norm(u)
        v = np.cross(d, u)
        t = np.linspace(0.0, length, max(2, int(length / 2)))[:, None]
        th = np.linspace(0.0, 2 * np.pi, max(8, int(2 * np.pi * r / 2)), endpoint=False)[None, :]
        pts = p + t[..., None] * d + r * (np.cos(th)[..., None] * u + np.sin(th)[..., None] * v)
        pts = pts.reshape(-1, 3)
        pts = pts[(pts >= 0).all(axis=1) & (pts < n).all(axis=1)]
        b = (pts // block).astype(np.int64)
        occ[b[:, 2], b[:, 1], b[:, 0]] = True
    z, y, x = np.nonzero(occ)
    return np.stack([x, y, z], axis=1).astype(np.int32)
