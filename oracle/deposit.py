"""Particle deposit: solid fraction, fluid fraction and drag force per finest node.

Test infrastructure (see ``oracle/__init__.py``).  The paper couples the
sediment to the fluid through a per-cell solid fraction eta that sets the
mixture fluid fraction eps = 1 - eta (Sec. 4, the tau_e = eps tau relaxation)
and through a drag force on the finest level (Sec. 5.4, computed during the
MPM grid update).  The MPM side is outside this path, so the fields come from
nearest-node particle counts with the readings below:

* the node of a particle at fine position p is floor(p) per axis, clamped
  into the domain;
* eta = min(eta_max, per_particle * count), eps = 1 - eta;
* F = (0, -kappa * eta, 0) while the particles move (drag toward the falling
  sediment along -y), F = 0 once they rest.

Plain numpy in float64; arrays indexed [z, y, x].
"""
import numpy as np


def node_counts(pos, shape_fine):
    """Particles per finest node: floor of each coordinate, clamped into the domain."""
    nz, ny, nx = shape_fine
    cnt = np.zeros((nz, ny, nx))
    for p in np.asarray(pos, dtype=np.float64):
        i = min(max(int(np.floor(p[0])), 0), nx - 1)
        j = min(max(int(np.floor(p[1])), 0), ny - 1)
        k = min(max(int(np.floor(p[2])), 0), nz - 1)
        cnt[k, j, i] += 1.0
    return cnt


def fields(pos, shape_fine, kappa=1e-4, eta_max=0.4, per_particle=0.25, moving=True):
    """(F[3, nz, ny, nx], eps[nz, ny, nx]) in float64 from particle positions (n, 3) (x, y, z)."""
    eta = np.minimum(eta_max, per_particle * node_counts(pos, shape_fine))
    F = np.zeros((3,) + tuple(shape_fine))
    if moving:
        F[1] = -kappa * eta
    return F, 1.0 - eta
