"""D3Q27 lattice, third-order Hermite reconstruction and moment projection.

Test infrastructure (see ``oracle/__init__.py``): plain FP64 restatement of
Sec. 3.1 of the paper, Eq. (rho_u_stress) and Eq. (three_order_f).

Velocity index convention of the oracle: i = (c_x+1) + 3 (c_y+1) + 9 (c_z+1),
so the rest velocity is i = 13 and the opposite of i is 26 - i.
"""
import itertools

import torch

CS2 = 1.0 / 3.0  # lattice speed of sound squared (Sec. 3.1, after Eq. rho_u_stress)

# D3Q27 velocities c_i in {-1,0,1}^3.  The paper names no velocity set; the
# seven third-order index triples it lists after Eq. (three_order_f) are exactly
# the non-degenerate third-order Hermite polynomials of D3Q27.
C = [(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1) for cx in (-1, 0, 1)]
Q = len(C)
OPP = [C.index((-c[0], -c[1], -c[2])) for c in C]

# Standard D3Q27 weights by the number of non-zero components of c_i.
_W_BY_CLASS = {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0}
W = [_W_BY_CLASS[sum(1 for a in c if a != 0)] for c in C]

# Moment rows of a field tensor M[10, ...].
RHO, UX, UY, UZ, SXX, SYY, SZZ, SXY, SXZ, SYZ = range(10)
S_INDEX = {(0, 0): SXX, (1, 1): SYY, (2, 2): SZZ,
           (0, 1): SXY, (1, 0): SXY, (0, 2): SXZ, (2, 0): SXZ,
           (1, 2): SYZ, (2, 1): SYZ}

# Third-order index triples listed after Eq. (three_order_f): xxy, xyy, xxz,
# xzz, yzz, yyz, xyz (x=0, y=1, z=2).
TRIPLES = [(0, 0, 1), (0, 1, 1), (0, 0, 2), (0, 2, 2), (1, 2, 2), (1, 1, 2), (0, 1, 2)]


def delta(a, b):
    return 1.0 if a == b else 0.0


def hermite2(c, a, b):
    """H^[2]_ab(c) = c_a c_b - c_s^2 delta_ab (Hermite basis, Sec. 3.1)."""
    return c[a] * c[b] - CS2 * delta(a, b)


def hermite3(c, a, b, g):
    """H^[3]_abg(c) = c_a c_b c_g - c_s^2 (delta_ab c_g + delta_ag c_b + delta_bg c_a)."""
    return c[a] * c[b] * c[g] - CS2 * (delta(a, b) * c[g] + delta(a, g) * c[b] + delta(b, g) * c[a])


def third_order_coeff(triple, mode="hermite"):
    """Weight of the term H^[3]_t Gamma_t in Eq. (three_order_f).

    The paper prints 1/(2 c_s^6) for every listed triple.  The full Hermite
    series sums over all ordered (a,b,g) with weight 1/(3! c_s^6); grouping the
    ordered triples by their sorted form gives (#permutations)/(6 c_s^6), which
    is 1/(2 c_s^6) for the six mixed triples and 1/c_s^6 for xyz.  ``hermite``
    uses the grouped series (the reconstruction then reproduces its own
    third-order moment); ``paper`` uses 1/(2 c_s^6) literally for all seven.
    """
    if mode == "paper":
        return 1.0 / (2.0 * CS2 ** 3)
    n_perm = len(set(itertools.permutations(triple)))
    return n_perm / (6.0 * CS2 ** 3)


def split_moments(M):
    """Return (rho, u[3], S[3][3]) views of a field tensor M[10, ...]."""
    rho = M[RHO]
    u = [M[UX], M[UY], M[UZ]]
    S = [[M[S_INDEX[(a, b)]] for b in range(3)] for a in range(3)]
    return rho, u, S


def gamma(S, u, a, b, g):
    """Gamma_abg = S_ab u_g + S_ag u_b + S_bg u_a - 2 u_a u_b u_g (Eq. three_order_f)."""
    return S[a][b] * u[g] + S[a][g] * u[b] + S[b][g] * u[a] - 2.0 * u[a] * u[b] * u[g]


def reconstruct(M, mode="hermite"):
    """f_i(M) for all 27 directions by Eq. (three_order_f).

    f_i = rho w_i [1 + c_i.u / c_s^2 + H2(c_i):S / (2 c_s^4)
                   + sum_t k_t H3_t(c_i) Gamma_t]
    where H2:S is the full double contraction sum_ab H2_ab S_ab and k_t is
    ``third_order_coeff(t, mode)``.  Returns a tensor of shape (27, ...).
    """
    rho, u, S = split_moments(M)
    f = torch.empty((Q,) + tuple(rho.shape), dtype=M.dtype)
    for i, c in enumerate(C):
        cu = sum(c[a] * u[a] for a in range(3))
        h2s = sum(hermite2(c, a, b) * S[a][b] for a in range(3) for b in range(3))
        third = 0.0
        for t in TRIPLES:
            h3 = hermite3(c, *t)
            if h3 != 0.0:
                third = third + third_order_coeff(t, mode) * h3 * gamma(S, u, *t)
        f[i] = rho * W[i] * (1.0 + cu / CS2 + h2s / (2.0 * CS2 ** 2) + third)
    return f


def project(f):
    """Moments of a distribution set (Eq. rho_u_stress without the force shift).

    Returns (rho, j[3], Pi[3][3]) with rho = sum f_i, j_a = sum c_ia f_i,
    Pi_ab = sum (c_ia c_ib - c_s^2 delta_ab) f_i.
    """
    rho = sum(f[i] for i in range(Q))
    j = [sum(C[i][a] * f[i] for i in range(Q)) for a in range(3)]
    Pi = [[sum(hermite2(C[i], a, b) * f[i] for i in range(Q)) for b in range(3)] for a in range(3)]
    return rho, j, Pi


def pack_moments(rho, u, S):
    """Assemble a field tensor M[10, ...] from rho, u[3] and symmetric S[3][3]."""
    return torch.stack([rho, u[0], u[1], u[2], S[0][0], S[1][1], S[2][2], S[0][1], S[0][2], S[1][2]])
