"""Pins for oracle functions that the dynamics tests leave loose.

* deposit: a hand-counted case (floor to the node, clamping, saturation, the
  sign and component of the drag);
* hierarchy flags and rebuild counts: set differences of the brute-force
  block sets of two consecutive hierarchies, and what each flag means for the
  children of the block;
* downward transfer: trilinear interpolation is exact on fields linear in x,
  y and z (rho, u and S^neq each linear), S^eq is formed from the
  interpolated u, and at s = 2 the coarse state is the temporal midpoint of
  rho, u and S^neq separately (a state that changes linearly in time);
* rebuild: on the analytic linear shear u_x = G y, whose post-collision
  S^neq_xy = -c_s^2 (tau_l - 1) 2^l G is known on every level (2^l: the level's
  lattice spacing in fine units), every node a rebuild creates or carries over
  equals the analytic field to rounding, in both consistent rescale readings;
  a node that both the finer and the coarser level could supply takes the
  finer level's value;
* reductions: momentum and kinetic energy with a non-zero velocity and a
  level-0 force shift, against hand sums over the owned nodes.
"""
import itertools

import numpy as np
import pytest
import torch

from oracle import deposit as dp
from oracle import hierarchy as hy
from oracle import multilevel as ml
from paper_2603_14982_gb300 import workloads as wl
from tests.test_oracle_multilevel import _as_set, brute


@pytest.fixture(autouse=True)
def _fp64_default_dtype():
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    yield
    torch.set_default_dtype(old)


# ------------------------------------------------------------------ deposit

def test_deposit_hand_counted():
    shape = (4, 4, 4)  # (nz, ny, nx)
    pos = np.array([[1.2, 2.7, 3.9],     # node (x 1, y 2, z 3)
                    [1.9, 2.1, 3.0],     # same node
                    [0.5, 0.5, 0.5],     # node (0, 0, 0)
                    [-2.0, 9.0, 1.5],    # clamped to (0, 3, 1)
                    [3.99, 0.0, 2.0]],   # node (3, 0, 2)
                   dtype=np.float32)
    F, eps = dp.fields(pos, shape)
    eta = np.zeros(shape)
    eta[3, 2, 1] = 0.4     # 2 x 0.25 saturates at 0.4
    eta[0, 0, 0] = 0.25
    eta[1, 3, 0] = 0.25
    eta[2, 0, 3] = 0.25
    assert np.array_equal(eps, 1.0 - eta)
    assert np.array_equal(F[0], np.zeros(shape)) and np.array_equal(F[2], np.zeros(shape))
    assert np.array_equal(F[1], -1e-4 * eta)
    F, eps = dp.fields(pos, shape, moving=False)
    assert not F.any() and np.array_equal(eps, 1.0 - eta)
    _, eps = dp.fields(pos, shape, eta_max=1.0, per_particle=0.1)
    assert eps[3, 2, 1] == 1.0 - 0.2 and eps[1, 3, 0] == 1.0 - 0.1


# ------------------------------------------------------------------ hierarchy flags

def _brute_flags(prev_sets, cur_sets, blocks, l, L):
    Hp, _, Sp, _ = prev_sets
    H, _, S, Bd = cur_sets
    out = []
    for b in map(tuple, blocks.tolist()):
        f = hy.BORDER if b in Bd[l] else hy.LEAF
        if b not in Sp[l]:
            f |= hy.NEW
        if b in H[l] and b not in Hp[l]:
            f |= hy.REFINE
        if b not in H[l] and b in Hp[l]:
            f |= hy.COARSEN
        out.append(f)
    return np.array(out, dtype=np.uint8)


def _falling(pos, t):
    return wl.fall(pos, t)


def _drifting(pos, t):
    # the cloud moves along the periodic x axis and falls: blocks are refined
    # ahead of it and coarsened behind it
    out = wl.fall(pos, t // 2)
    out[:, 0] = np.mod(out[:, 0] + np.float32(t), np.float32(128.0))
    return out


@pytest.mark.parametrize("motion", [_falling, _drifting])
def test_flags_and_counts_against_brute_force_sets(motion):
    ext, B, L, per = (128, 128, 128), 8, 3, (True, False, True)
    pos = wl.particle_cloud(128, count=4000, seed=7)
    prev, prev_sets = None, None
    seen = 0
    for t in range(0, 132, 12):
        p = motion(pos, t)
        h = hy.from_particles(p, ext, B, L, per)
        O0 = {(int(q[0]) // 8, int(q[1]) // 8, int(q[2]) // 8) for q in p}
        sets = brute(O0, ext, B, L, per)
        if prev is not None:
            for l in range(L):
                f = h.flags(l, prev)
                assert np.array_equal(f, _brute_flags(prev_sets, sets, h.blocks(l), l, L)), (t, l)
                seen |= int(np.bitwise_or.reduce(f)) if len(f) else 0
                # what the flags mean for the children of a block
                if l > 0:
                    kids_now = hy.parent(h.stored[l - 1] | h.I[l - 1])
                    kids_before = hy.parent(prev.stored[l - 1] | prev.I[l - 1])
                    z, y, x = np.nonzero(h.stored[l])
                    ref = (f & hy.REFINE) != 0
                    coa = (f & hy.COARSEN) != 0
                    assert (kids_now[z, y, x][ref]).all() and not (kids_before[z, y, x][ref]).any()
                    assert not (kids_now[z, y, x][coa]).any() and (kids_before[z, y, x][coa]).all()
            Hp, _, Sp, _ = prev_sets
            H, _, S, _ = sets
            refined = sum(len(H[l] - Hp[l]) for l in range(L))
            coarsened = sum(len(Hp[l] - H[l]) for l in range(L))
            deleted = sum(len(Sp[l] - S[l]) for l in range(L))
            assert h.counts(prev) == (refined, coarsened, deleted)
        prev, prev_sets = h, sets
    # the drifting cloud exercises every flag bit (the falling one never refines:
    # it starts at the floor)
    want = hy.LEAF | hy.BORDER | hy.NEW | hy.COARSEN | (hy.REFINE if motion is _drifting else 0)
    assert seen == want


# ------------------------------------------------------------------ downward transfer

def _linear(coef, X, Y, Z):
    c0, cx, cy, cz = coef
    return c0 + cx * X + cy * Y + cz * Z


# dyadic coefficients: every product and 1/8-weighted sum is exact in binary
RHO = (1.0, 2.0 ** -9, -(2.0 ** -10), 3 * 2.0 ** -11)
U = [(0.03, 2.0 ** -10, 0.0, -(2.0 ** -11)), (-0.02, 0.0, 2.0 ** -10, 2.0 ** -12),
     (0.01, -(2.0 ** -12), 2.0 ** -11, 0.0)]
SNEQ = [(1e-4 * (r + 1), 2.0 ** -16 * (r - 2), 2.0 ** -17 * (3 - r), 2.0 ** -18) for r in range(6)]


def _state(coefs, X, Y, Z):
    rho = torch.as_tensor(_linear(coefs[0], X, Y, Z))
    u = [torch.as_tensor(_linear(c, X, Y, Z)) for c in coefs[1]]
    s = [torch.as_tensor(_linear(c, X, Y, Z)) for c in coefs[2]]
    return rho, u, s


def _expected(rho, u, sneq, k):
    eq = [u[0] * u[0], u[1] * u[1], u[2] * u[2], u[0] * u[1], u[0] * u[2], u[1] * u[2]]
    return torch.stack([rho] + list(u) + [k * sneq[r] + eq[r] for r in range(6)])


def test_interpolate_down_exact_on_linear_fields():
    nc = (6, 5, 7)  # coarse nodes (z, y, x)
    cz, cy, cx = np.meshgrid(*(np.arange(n) for n in nc), indexing="ij")
    Mc = _state((RHO, U, SNEQ), 2.0 * cx, 2.0 * cy, 2.0 * cz)   # coarse node i sits at fine 2 i
    # every fine node whose stencil stays inside the coarse grid (no clamp, no wrap)
    pz, py, px = np.meshgrid(*(np.arange(2 * n - 1) for n in nc), indexing="ij")
    nodes = (pz.ravel(), py.ravel(), px.ravel())
    k = 0.37
    got = ml.interpolate_down(Mc, nodes, (False, False, False), k)
    want = _expected(*_state((RHO, U, SNEQ), px.ravel() * 1.0, py.ravel() * 1.0, pz.ravel() * 1.0), k)
    assert (got - want).abs().max() < 1e-15
    # S^eq from the interpolated u, not the interpolated coarse u u: they
    # differ at odd fine indices by the curvature of u u
    uu_c = Mc[1][0] * Mc[1][0]
    avg_uu = 0.5 * (uu_c[0, 0, 0] + uu_c[0, 0, 1])
    assert abs(float(avg_uu) - float(want[1][1]) ** 2) > 1e-7


def _two_level_machine(tau0=0.9):
    ext, B, L = (48, 48, 48), 4, 2
    O0 = np.zeros(hy.block_dims(ext, B, 0), bool)
    O0[5:7, 5:7, 5:7] = True
    h = hy.Hierarchy(O0, ext, B, L, (True, True, True))
    return ml.MultiLevel(h, tau0)


@pytest.mark.parametrize("s", [1, 2])
def test_downward_transfer_temporal_midpoint(s):
    m = _two_level_machine()
    X1, Y1, Z1 = m.node_positions(1)
    old = (RHO, U, SNEQ)
    # the new coarse state: every field moved linearly in time, u by O(1e-2) so
    # that averaging S instead of S^neq would show
    new = ((RHO[0] + 2e-3, RHO[1], RHO[2], RHO[3]),
           [(c[0] + 0.02 * (a + 1), c[1], c[2], c[3]) for a, c in enumerate(U)],
           [(c[0] - 3e-5, c[1], c[2], c[3]) for c in SNEQ])
    m.set_level(0, wl.rest_field(m.shape[0]))
    m.set_level(1, ml.join_neq(*_state(new, X1, Y1, Z1), 1.0).numpy())
    prev = ml.join_neq(*_state(old, X1, Y1, Z1), 1.0)
    prev[:, ~m.stored[1]] = float("nan")
    m.buf[1][1 - m.cur[1]] = prev
    m.downward_transfer(1, s)
    nodes = m.down[0]
    assert len(nodes[0]) > 0
    pz, py, px = (n.astype(np.float64) for n in nodes)
    ro, uo, so = _state(old, px, py, pz)
    rn, un, sn = _state(new, px, py, pz)
    _, k_down = m.k_updown(0)
    if s == 1:
        want = _expected(ro, uo, so, k_down)
    else:
        want = _expected(0.5 * (ro + rn), [0.5 * (uo[a] + un[a]) for a in range(3)],
                         [0.5 * (so[r] + sn[r]) for r in range(6)], k_down)
    got = m.current(0)[:, nodes[0], nodes[1], nodes[2]]
    assert (got - want).abs().max() < 1e-15


# ------------------------------------------------------------------ rebuild

G = 2.0 ** -12  # du_x/dy per fine node


def _shear_level(m, l, mode, drho=0.0):
    """Analytic linear shear on level l: rho = 1 + drho + 2^-12 (y - y0),
    u_x = G (y - y0) with y0 the middle of the domain, S^neq_xy =
    -c_s^2 (tau_l - 1) 2^l G (post) or -c_s^2 tau_l 2^l G (pre)."""
    X, Y, Z = m.node_positions(l)
    y0 = m.h.extent[1] / 2.0
    ux = G * (Y - y0)
    rho = 1.0 + drho + 2.0 ** -12 * (Y - y0)
    t = m.tau[l] - 1.0 if mode == "post" else m.tau[l]
    sxy = -t * (2 ** l) * G / 3.0
    z0 = np.zeros_like(ux)
    return wl._pack(rho, ux, z0, z0, ux * ux, z0, z0, sxy + z0, z0, z0)


def _hier(ext, B, L, cells):
    O0 = np.zeros(hy.block_dims(ext, B, 0), bool)
    for c in cells:
        O0[c] = True
    return hy.Hierarchy(O0, ext, B, L, (True, True, True))


@pytest.mark.parametrize("mode", ["post", "pre"])
@pytest.mark.parametrize("L", [2, 3])
def test_rebuild_carries_the_analytic_shear(mode, L):
    if L == 2:
        ext, B = (32, 64, 32), 4
        h0 = _hier(ext, B, L, [(3, 7, 3), (3, 8, 3)])
        h1 = _hier(ext, B, L, [(4, 8, 5), (4, 9, 5), (5, 9, 5)])
    else:
        ext, B = (64, 128, 64), 4
        h0 = _hier(ext, B, L, [(7, 15, 7), (7, 16, 7)])
        h1 = _hier(ext, B, L, [(8, 17, 10), (8, 18, 10), (9, 18, 10)])
    assert all(len(h.blocks(l)) > 0 for h in (h0, h1) for l in range(L))
    m = ml.MultiLevel(h0, 1.2 if mode == "post" else 0.8, rescale=mode)
    for l in range(L):
        m.set_level(l, _shear_level(m, l, mode))
    m.rebuild(h1)
    new_nodes = 0
    for l in range(L):
        st = m.stored[l]
        want = torch.as_tensor(_shear_level(m, l, mode))[:, st]
        got = m.current(l)[:, st]
        assert (got - want).abs().max() < 1e-15, l
        new_nodes += int((st & ~torch.as_tensor(h0.stored_nodes(l))).sum())
    assert new_nodes > 0


def test_rebuild_prefers_the_finer_source():
    """Levels offset in rho by 0, 1e-3, 2e-3: nodes new at level 1 whose
    coincident level-0 node was stored (and not an interface node) take the
    level-0 value (upward rule) rather than the level-2 value."""
    ext, B, L = (64, 128, 64), 4, 3
    h0 = _hier(ext, B, L, [(z, y, x) for z in (7, 8) for y in (15, 16) for x in (7, 8)])
    h1 = _hier(ext, B, L, [(7, 21, 7)])
    assert all(len(h.blocks(l)) > 0 for h in (h0, h1) for l in range(L))
    m = ml.MultiLevel(h0, 1.2)
    for l in range(L):
        m.set_level(l, _shear_level(m, l, "post", drho=1e-3 * l))
    m.rebuild(h1)
    new1 = torch.as_tensor(h1.stored_nodes(1) & ~h0.stored_nodes(1))
    fine_src = torch.as_tensor((h0.stored_nodes(0) & ~h0.down_nodes(0))[0::2, 0::2, 0::2])
    cat = new1 & fine_src
    assert int(cat.sum()) > 0
    want = torch.as_tensor(_shear_level(m, 1, "post", drho=0.0))
    assert (m.current(1)[:, cat] - want[:, cat]).abs().max() < 1e-15


# ------------------------------------------------------------------ reductions

def test_reduce_momentum_and_energy_by_hand():
    ext, L = (64, 64, 64), 3
    O0 = np.zeros(hy.block_dims(ext, 8, 0), bool)
    O0[2, 2, 2] = True
    h = hy.Hierarchy(O0, ext, 8, L, (True, True, True))
    F = (0.02, 0.0, 0.01)
    m = ml.MultiLevel(h, 0.9, force=F)
    rho0, u0s = 1.25, (0.1, 0.02, 0.0)          # level 0: stored u' = u + F / (2 rho)
    rho1, u1 = 0.8, (0.0, 0.05, 0.0)
    for l in range(L):
        X, _, _ = m.node_positions(l)
        r, u = (rho0, u0s) if l == 0 else (rho1, u1)
        m.set_level(l, wl.equilibrium_field(np.full_like(X, r), *(np.full_like(X, v) for v in u)))
    n = [int(h.owned_nodes(l).sum()) for l in range(L)]
    assert sum(n[l] * 8 ** l for l in range(L)) == 64 ** 3
    vc = n[1] * 8 + n[2] * 64  # fine-equivalent volume of the coarse levels
    up = (0.1 - 0.02 / 2.5, 0.02, -0.01 / 2.5)  # physical level-0 velocity
    r = m.reduce()
    want = [rho0 * n[0] + rho1 * vc,
            rho0 * up[0] * n[0],
            rho0 * up[1] * n[0] + rho1 * 0.05 * vc,
            rho0 * up[2] * n[0],
            0.5 * rho0 * (up[0] ** 2 + up[1] ** 2 + up[2] ** 2) * n[0] + 0.5 * rho1 * 0.05 ** 2 * vc,
            rho0 * n[0],
            rho1 * vc]
    for a, b in zip(r, want):
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b))
