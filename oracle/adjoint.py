"""Reverse-mode gradient of the single-level step with respect to the body force.

Test infrastructure (see ``oracle/__init__.py``).  The paper has no adjoint;
this module differentiates the oracle's own forward model (``single_level``)
so the GPU adjoint can be checked against it:

* ``gradient``: dL/dF by reverse-mode automatic differentiation of the FP64
  forward run (a library primitive applied to the plain forward code), with
  segment checkpointing so large runs fit in memory;
* ``complex_step``: the directional derivative Im L(F + i h e) / h with
  h = 1e-30, exact to rounding because the forward uses only + - * / and
  branches that do not depend on the values;
* ``outlet_kinetic_energy``: the loss of the obstacle-channel workload,
  L = 1/2 sum over the last x-plane of rho |u|^2 with the physical velocity
  u = u' - F/(2 rho);
* ``ml_gradient`` / ``ml_complex_step``: the same two derivatives of the
  multi-level advance (Algorithm 1 of ``multilevel``: sub-cycled steps, the
  downward transfer with its temporal midpoint and the upward transfer with
  their S^neq rescaling), for the linear loss L = sum_l <W_l, M_l> over the
  stored nodes of every level after the run.
"""
import torch
from torch.utils.checkpoint import checkpoint

from . import multilevel as ml
from . import single_level as sl

# Rest state (rho = 1, u = 0, S = 0): the finite value the multi-level
# derivatives give the nodes a level does not store.
REST = [1.0] + [0.0] * 9


def outlet_kinetic_energy(M, F):
    """L = 1/2 sum_{x = nx-1} rho |u|^2, physical u (analytic in M and F: no abs/conj)."""
    u = sl.physical_velocity(M, F)
    rho = M[0]
    ke = 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
    return ke[:, :, -1].sum()


def run_forward(M0, F, steps, tau, periodic, solid=None, mode="hermite", ckpt_every=None):
    """Forward run of ``steps`` single-level steps with force field F (3, nz, ny, nx)."""
    blocked = sl.blocked_sources(tuple(M0.shape[1:]), periodic, solid)

    def seg(M, Fv, n):
        for _ in range(n):
            M = sl.step(M, tau, force=Fv, periodic=periodic, solid=solid, mode=mode, blocked=blocked)
        return M

    M = M0
    if ckpt_every is None or not F.requires_grad:
        return seg(M, F, steps)
    done = 0
    while done < steps:
        n = min(ckpt_every, steps - done)
        M = checkpoint(seg, M, F, n, use_reentrant=False)
        done += n
    return M


def gradient(M0, F, steps, tau, periodic, solid=None, mode="hermite", ckpt_every=None):
    """(L, dL/dF) of the outlet kinetic energy after ``steps`` steps, FP64."""
    Fv = F.detach().clone().requires_grad_(True)
    M = run_forward(M0, Fv, steps, tau, periodic, solid, mode, ckpt_every)
    L = outlet_kinetic_energy(M, Fv)
    (g,) = torch.autograd.grad(L, Fv)
    return L.detach(), g


def complex_step(M0, F, steps, tau, periodic, direction, solid=None, mode="hermite", h=1e-30):
    """d/dh L(F + h * direction) at h = 0 by the complex step, exact to rounding."""
    Mc = M0.to(torch.complex128)
    Fc = F.to(torch.complex128) + 1j * h * direction.to(torch.complex128)
    M = run_forward(Mc, Fc, steps, tau, periodic, solid, mode)
    return (outlet_kinetic_energy(M, Fc).imag / h).item()


def ml_forward(hier, tau0, M0, F, n_coarse, rescale="post", mode="hermite", dtype=torch.float64):
    """Dense stored moments of every level after ``n_coarse`` coarse steps of
    Algorithm 1 from the dense per-level fields M0 with the level-0 force
    field F (3, nz, ny, nx).  Nodes a level does not store hold ``REST``."""
    m = ml.MultiLevel(hier, tau0, mode=mode, rescale=rescale, force=F)
    for l in range(m.L):
        m.set_level(l, M0[l], fill=REST, dtype=dtype)
    for _ in range(n_coarse):
        m.coarse_step()
    return [m.current(l) for l in range(m.L)], m


def ml_weighted_sum(Ms, W):
    """L = sum_l <W_l, M_l>; W_l is zero at the nodes level l does not store."""
    return sum((torch.as_tensor(W[l]) * Ms[l]).sum() for l in range(len(Ms)))


def ml_gradient(hier, tau0, M0, F, n_coarse, W, rescale="post", mode="hermite"):
    """(L, dL/dF) of ``ml_weighted_sum`` after the multi-level run, FP64."""
    Fv = torch.as_tensor(F, dtype=torch.float64).detach().clone().requires_grad_(True)
    Ms, _ = ml_forward(hier, tau0, M0, Fv, n_coarse, rescale, mode)
    L = ml_weighted_sum(Ms, W)
    (g,) = torch.autograd.grad(L, Fv)
    return L.detach(), g


def ml_complex_step(hier, tau0, M0, F, n_coarse, W, direction, rescale="post", mode="hermite", h=1e-30):
    """d/dh L(F + h * direction) at h = 0 for the multi-level run, by the complex step."""
    Fc = torch.as_tensor(F).to(torch.complex128) + 1j * h * torch.as_tensor(direction).to(torch.complex128)
    Ms, _ = ml_forward(hier, tau0, M0, Fc, n_coarse, rescale, mode, dtype=torch.complex128)
    return (ml_weighted_sum(Ms, W).imag / h).item()
