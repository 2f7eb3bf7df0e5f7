"""The coupled finest-level step of Fig. 4: streaming only (S), force exchange
(Ex), collision (C).

Test infrastructure (see ``oracle/__init__.py``).  Sec. 5.4 describes one
LBM-MPM advance: after the streaming step at level 0 the fluid and sediment
fractions and the drag are computed and fed into the collision step, and the
MPM side runs once every few LBM steps.  Readings of what the paper leaves open:

* the drag on the fluid is linear in the relative velocity,
  F = kappa * eta * (v_p - u*), with eta = 1 - eps the solid fraction, v_p
  the sediment velocity and u* = j* / rho* the velocity of the streamed
  populations (the paper cites the Di Felice law without printing it; kappa
  stands for its drag coefficient);
* the force of an exchange step is kept for the steps up to the next one;
* nodes that keep their moments (solid, interface) feel no drag (F = 0).
"""
import torch

from . import lattice as lat
from . import single_level as sl


def drag(fstar, eps, vp, kappa):
    """F[3, ...] = kappa (1 - eps) (vp - j*/rho*) from streamed populations."""
    rho, j, _ = lat.project(fstar)
    eta = 1.0 - (eps if eps is not None else torch.ones_like(rho))
    return torch.stack([kappa * eta * (float(vp[a]) - j[a] / rho) for a in range(3)])


def coupled_step(M, tau, eps, vp, kappa, periodic=(True, True, True), solid=None, mode="hermite",
                 update=None, blocked=None):
    """S, Ex, C: returns (M', F) with F the exchanged drag (zero where M is kept)."""
    fstar = sl.stream(M, periodic, solid, mode, blocked)
    F = drag(fstar, eps, vp, kappa)
    keep = torch.zeros(tuple(M.shape[1:]), dtype=torch.bool)
    if solid is not None:
        keep |= solid
    if update is not None:
        keep |= ~update
    F = torch.where(keep.unsqueeze(0), torch.zeros_like(F), F)
    Mn, _ = sl.collide(fstar, tau, force=F, eps=eps)
    return torch.where(keep.unsqueeze(0), M, Mn), F


def run_coupled(M, n_steps, tau, eps, vp, kappa, every, periodic=(True, True, True), solid=None, mode="hermite"):
    """n_steps level steps; steps 0, every, 2 every, ... exchange the drag, the
    others use the last exchanged force.  Returns (M, F)."""
    blocked = sl.blocked_sources(tuple(M.shape[1:]), periodic, solid)
    F = None
    for i in range(n_steps):
        if i % every == 0:
            M, F = coupled_step(M, tau, eps, vp, kappa, periodic, solid, mode, blocked=blocked)
        else:
            M = sl.step(M, tau, force=F, eps=eps, periodic=periodic, solid=solid, mode=mode, blocked=blocked)
    return M, F
