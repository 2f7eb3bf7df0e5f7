"""Pins for the oracle's lattice, reconstruction and single-level step.

Each test checks the FP64 oracle against something the paper or the
mathematics fixes independently of the oracle's own code: lattice isotropy,
the Hermite projection identities of Eq. (three_order_f), exact conservation,
Galilean/symmetry invariances, closed-form Taylor-Green decay, the steady
Poiseuille profile and the transient square-duct series.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lattice as lat
from oracle import single_level as sl
from paper_2603_14982_gb300 import workloads as wl



@pytest.fixture(autouse=True)
def _fp64_default_dtype():
    """FP64 default dtype for the oracle's tensors, restored afterwards: the
    GPU tests collected in the same session must keep torch's float32 default."""
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    yield
    torch.set_default_dtype(old)


def T(a):
    return torch.tensor(a, dtype=torch.float64)


# ---------------------------------------------------------------- lattice

def test_weights_isotropy():
    """D3Q27 weights: sum 1, second moment c_s^2 delta, isotropic fourth moment."""
    cs2 = 1.0 / 3.0
    assert abs(sum(lat.W) - 1.0) < 1e-15
    for a in range(3):
        for b in range(3):
            m2 = sum(w * c[a] * c[b] for w, c in zip(lat.W, lat.C))
            assert abs(m2 - cs2 * (a == b)) < 1e-15
            for g in range(3):
                for d in range(3):
                    m4 = sum(w * c[a] * c[b] * c[g] * c[d] for w, c in zip(lat.W, lat.C))
                    iso = cs2 ** 2 * ((a == b) * (g == d) + (a == g) * (b == d) + (a == d) * (b == g))
                    assert abs(m4 - iso) < 1e-15
    assert lat.C[13] == (0, 0, 0)
    assert all(lat.C[lat.OPP[i]] == tuple(-x for x in lat.C[i]) for i in range(27))


def _moment(f, poly):
    return sum(poly(lat.C[i]) * f[i] for i in range(27))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_projection_identities(seed):
    """The reconstruction reproduces the moments it was built from.

    sum f = rho, sum c f = rho u, sum H2 f = rho S, and, with the Hermite
    coefficients, sum H3_t f = rho Gamma_t for all seven triples.
    """
    M = T(wl.random_field((3, 4, 5), seed, du=0.05, drho=0.05, dneq=0.01))
    rho, u, S = lat.split_moments(M)
    f = lat.reconstruct(M, "hermite")
    tol = 1e-14
    assert (_moment(f, lambda c: 1.0) - rho).abs().max() < tol
    for a in range(3):
        assert (_moment(f, lambda c: c[a]) - rho * u[a]).abs().max() < tol
        for b in range(3):
            h2 = _moment(f, lambda c: c[a] * c[b] - (a == b) / 3.0)
            assert (h2 - rho * S[a][b]).abs().max() < tol
    for t in lat.TRIPLES:
        a, b, g = t
        h3 = _moment(f, lambda c: c[a] * c[b] * c[g]
                     - ((a == b) * c[g] + (a == g) * c[b] + (b == g) * c[a]) / 3.0)
        gam = S[a][b] * u[g] + S[a][g] * u[b] + S[b][g] * u[a] - 2 * u[a] * u[b] * u[g]
        assert (h3 - rho * gam).abs().max() < tol


def test_paper_literal_xyz_coefficient_halves_third_moment():
    """With the coefficient printed for xyz (1/(2 c_s^6)) the xyz third moment is half."""
    M = T(wl.random_field((2, 2, 2), 4, du=0.05, dneq=0.01))
    rho, u, S = lat.split_moments(M)
    f = lat.reconstruct(M, "paper")
    h3 = _moment(f, lambda c: c[0] * c[1] * c[2])
    gam = S[0][1] * u[2] + S[0][2] * u[1] + S[1][2] * u[0] - 2 * u[0] * u[1] * u[2]
    assert (h3 - 0.5 * rho * gam).abs().max() < 1e-15


def test_rest_state_is_weights():
    rho = T(np.full((2, 2, 2), 1.3))
    z = torch.zeros_like(rho)
    M = lat.pack_moments(rho, [z, z, z], [[z] * 3] * 3)
    f = lat.reconstruct(M)
    for i in range(27):
        assert torch.allclose(f[i], 1.3 * lat.W[i] * torch.ones_like(rho), rtol=0, atol=1e-16)


def test_equilibrium_matches_second_order_feq_up_to_third_order_terms():
    """With S = u u the reconstruction equals Eq. (lbe_feq) plus terms cubic in u."""
    u0 = 1e-3
    M = T(wl.equilibrium_field(np.ones((1, 1, 1)), np.full((1, 1, 1), u0),
                               np.full((1, 1, 1), -0.5 * u0), np.full((1, 1, 1), 0.25 * u0)))
    f = lat.reconstruct(M)
    u = (u0, -0.5 * u0, 0.25 * u0)
    uu = sum(x * x for x in u)
    for i, c in enumerate(lat.C):
        cu = sum(c[a] * u[a] for a in range(3))
        feq = lat.W[i] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
        assert abs(f[i].item() - feq) < 30 * u0 ** 3


# ---------------------------------------------------------------- one step

def test_mass_conserved_periodic_and_walls():
    M = T(wl.random_field((6, 8, 10), 11))
    m0 = M[0].sum()
    M1 = sl.run(M, 5, 0.6)
    assert abs((M1[0].sum() - m0) / m0) < 1e-13
    solid = torch.zeros((6, 8, 10), dtype=torch.bool)
    solid[2:4, 3:5, 4:7] = True
    M = torch.where(solid.unsqueeze(0), T(wl.rest_field((6, 8, 10))), M)
    m0 = M[0].sum()
    M1 = sl.run(M, 5, 0.7, periodic=(True, False, False), solid=solid)
    assert abs((M1[0].sum() - m0) / m0) < 1e-13


def test_momentum_grows_by_total_force():
    """Periodic box: sum rho u' (stored) increases by exactly sum F per step."""
    shape = (4, 6, 8)
    M = T(wl.random_field(shape, 12))
    F = T(wl.noisy_force(shape, seed=3, mean=(1e-4, -2e-4, 5e-5), sigma=1e-4))
    for _ in range(3):
        p0 = [(M[0] * M[1 + a]).sum() for a in range(3)]
        M = sl.step(M, 0.7, force=F)
        for a in range(3):
            assert abs((M[0] * M[1 + a]).sum() - p0[a] - F[a].sum()) < 1e-15 * M[0].numel() + 1e-14


def test_uniform_flow_is_preserved():
    shape = (4, 4, 4)
    u = (0.05, 0.02, -0.01)
    M = T(wl.equilibrium_field(np.ones(shape), *(np.full(shape, x) for x in u)))
    M1 = sl.run(M, 4, 0.55)
    assert (M1 - M).abs().max() < 1e-15


def test_uniform_force_on_uniform_flow():
    """u(t) = u0 + t F / rho for the physical velocity, exactly."""
    shape = (2, 2, 2)
    F = (1e-4, -3e-5, 2e-5)
    M = T(wl.equilibrium_field(np.ones(shape), np.full(shape, 0.01), np.zeros(shape), np.zeros(shape)))
    M = sl.step(M, 0.8, force=F)       # after the first step the stored u carries the F/2 shift
    u1 = [x.clone() for x in sl.physical_velocity(M, F)]
    for t in range(1, 6):
        M = sl.step(M, 0.8, force=F)
        u = sl.physical_velocity(M, F)
        for a in range(3):
            assert (u[a] - (u1[a] + t * F[a])).abs().max() < 1e-15


def test_mirror_symmetry_x():
    """Reflecting x (u_x, S_xy, S_xz change sign) commutes with the step."""
    M = T(wl.random_field((5, 6, 7), 21))

    def mirror(A):
        B = torch.flip(A, dims=(3,)).clone()
        for r in (1, 7, 8):
            B[r] = -B[r]
        return B

    F = T(wl.noisy_force((5, 6, 7), seed=9, mean=(0, 0, 0), sigma=1e-4))
    Fm = torch.flip(F, dims=(3,)).clone()
    Fm[0] = -Fm[0]
    a = sl.run(M, 3, 0.65, force=F, periodic=(False, True, False))
    b = sl.run(mirror(M), 3, 0.65, force=Fm, periodic=(False, True, False))
    assert (mirror(a) - b).abs().max() < 1e-15


def test_axis_permutation_covariance():
    """Cycling the axes (x->y->z->x) of the input cycles the output."""
    M = T(wl.random_field((6, 6, 6), 22))

    def cyc(A):
        # new field G(x', y', z') with x'=z, y'=x, z'=y: arrays are [z,y,x]
        B = A.permute(0, 2, 3, 1).clone()          # [.., y, x, z] -> indexes (z'=y, y'=x, x'=z)
        rho, ux, uy, uz, sxx, syy, szz, sxy, sxz, syz = B
        return torch.stack([rho, uz, ux, uy, szz, sxx, syy, sxz, syz, sxy])

    a = sl.run(M, 3, 0.6, periodic=(True, False, True))
    b = sl.run(cyc(M), 3, 0.6, periodic=(True, True, False))
    assert (cyc(a) - b).abs().max() < 1e-15


def test_mixture_tau_scaling():
    """eps*tau enters only as the product: eps = 0.5, tau = 1.2 equals tau = 0.6."""
    M = T(wl.random_field((4, 4, 4), 23))
    a = sl.step(M, 0.6)
    b = sl.step(M, 1.2, eps=torch.full((4, 4, 4), 0.5))
    assert (a - b).abs().max() < 1e-16


def test_rest_with_walls_and_obstacle_stays_at_rest():
    shape = (8, 8, 8)
    solid = T(wl.obstacle_mask(8, 3, 5)).bool()
    M = T(wl.rest_field(shape))
    M1 = sl.run(M, 3, 0.7, periodic=(True, False, False), solid=solid)
    assert (M1 - M).abs().max() < 1e-14


# ---------------------------------------------------------------- closed forms

def _nu_eff_tgv2d(n, tau, u0, steps):
    M0 = T(wl.taylor_green_2d(n, 1, u0))
    M1 = sl.run(M0, steps, tau)
    k = 2 * math.pi / n
    return -math.log(sl.kinetic_energy(M1) / sl.kinetic_energy(M0)) / (4 * k * k * steps)


def test_taylor_green_2d_viscosity_second_order():
    """z-invariant TGV decays as exp(-4 nu k^2 t), nu = c_s^2 (tau - 1/2);
    the effective viscosity error falls ~4x from n=16 to n=32 (diffusive scaling)."""
    tau = 0.6
    nu = (tau - 0.5) / 3.0
    e16 = _nu_eff_tgv2d(16, tau, 0.05, 100) / nu - 1
    e32 = _nu_eff_tgv2d(32, tau, 0.025, 400) / nu - 1
    assert abs(e16) < 0.03 and abs(e32) < 0.008
    assert 3.5 < e16 / e32 < 4.5


def test_taylor_green_3d_decay():
    """3D TGV, 32^3, tau = 0.6.  At U0 = 0.05 (Re ~ 8) KE(100)/KE(0) is within a few
    percent of exp(-6 nu k^2 t) (nonlinear transfer and the start-up transient of
    an initial state without non-equilibrium stress).  At U0 = 0.001 the flow is
    linear and the decay rate over t in [50, 100] is 6 nu k^2 to the O(k^2)
    lattice error."""
    tau, n, t = 0.6, 32, 100
    nu, k = (tau - 0.5) / 3, 2 * math.pi / n
    M0 = T(wl.taylor_green_3d(n, 0.05))
    r = (sl.kinetic_energy(sl.run(M0, t, tau)) / sl.kinetic_energy(M0)).item()
    assert abs(r / math.exp(-6 * nu * k * k * t) - 1) < 0.05
    M = sl.run(T(wl.taylor_green_3d(n, 0.001)), 50, tau)
    ke50 = sl.kinetic_energy(M).item()
    ke100 = sl.kinetic_energy(sl.run(M, 50, tau)).item()
    rate = -math.log(ke100 / ke50) / 50
    assert abs(rate / (6 * nu * k * k) - 1) < 0.01


def test_poiseuille_steady_profile():
    """Plane channel between half-way bounce-back walls: u = g/(2 nu) y'(W - y'), y' = y + 1/2."""
    W, g, tau = 16, 1e-6, 0.8
    nu = (tau - 0.5) / 3
    M = T(wl.rest_field((1, W, 1)))
    M = sl.run(M, int(8 * W * W / nu / math.pi ** 2), tau, force=(g, 0, 0), periodic=(True, False, True))
    u = sl.physical_velocity(M, (g, 0, 0))[0][0, :, 0]
    y = torch.arange(W) + 0.5
    ua = g / (2 * nu) * y * (W - y)
    assert ((u - ua).abs().max() / ua.max()) < 2e-3


def duct_series(W, g, nu, t, y, z, terms=199):
    """Transient square duct from rest (walls at -1/2 and W-1/2):
    u(y,z,t) = sum_{m,n odd} 16 g / (pi^2 m n nu lam) (1 - exp(-nu lam t)) sin(m pi y'/W) sin(n pi z'/W)."""
    yb, zb = y + 0.5, z + 0.5
    u = np.zeros(np.broadcast(yb, zb).shape)
    for m in range(1, terms + 1, 2):
        for n in range(1, terms + 1, 2):
            lam = math.pi ** 2 * (m * m + n * n) / W ** 2
            u += (16 * g / (math.pi ** 2 * m * n * nu * lam) * (1 - math.exp(-nu * lam * t))
                  * np.sin(m * math.pi * yb / W) * np.sin(n * math.pi * zb / W))
    return u


def test_square_duct_transient_series():
    """The force-driven duct from rest (periodic x, walls in y and z) follows the series."""
    W, g, tau, t = 16, 1e-6, 0.8, 300
    nu = (tau - 0.5) / 3
    M = T(wl.rest_field((W, W, 1)))
    M = sl.run(M, t, tau, force=(g, 0, 0), periodic=(True, False, False))
    u = sl.physical_velocity(M, (g, 0, 0))[0][:, :, 0].numpy()
    z, y = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    ua = duct_series(W, g, nu, t, y, z)
    assert np.abs(u - ua).max() / ua.max() < 1e-2
