"""One single-level pull-stream + moment-space collision step on a dense grid.

Test infrastructure (see ``oracle/__init__.py``).  Follows the paper's operator
splitting of Eq. (lbe_normalized): every node pulls f_i*(x) = f_i(M(x - c_i))
reconstructed by Eq. (three_order_f) from its neighbour's stored moments
(Sec. 3.1 "Collision and Streaming"), projects them to rho*, rho* u*, rho* S*
(Eq. rho_u_stress), and applies a BGK collision in Hermite-moment space with a
Guo body force and the mixture relaxation time eps*tau (Sec. 4, the evolution
equation with -(f - f^eq)/(eps tau)).

Readings of passages the paper leaves open:
* the stored moment set is the POST-collision one, so the stored velocity is
  u' = u + F/(2 rho) where u = (j* + F/2)/rho* is the physical velocity of
  Eq. (rho_u_stress);
* the collision relaxes rho* S* towards rho* u u with rate 1/(eps tau) and adds
  the Guo source (1 - 1/(2 eps tau)) (u F + F u);
* walls on non-periodic axes sit half a node outside the first/last node and
  use half-way bounce-back f_i*(x) = f_opp(i)(M(x)); solid nodes are frozen.
"""
import torch

from . import lattice as lat


def _as_components(force, shape, dtype):
    if force is None:
        return [torch.zeros(shape, dtype=dtype) for _ in range(3)]
    if isinstance(force, torch.Tensor) and force.dim() == 4:
        return [force[0], force[1], force[2]]
    return [torch.full(shape, float(force[a]), dtype=dtype) for a in range(3)]


def blocked_sources(shape, periodic, solid=None):
    """For each direction i, the nodes x whose pull source x - c_i is a wall or solid.

    ``periodic`` is (px, py, pz).  Returns a list of 27 bool tensors (nz, ny, nx).
    """
    nz, ny, nx = shape
    coord = torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx), indexing="ij")
    coord_xyz = (coord[2], coord[1], coord[0])
    extent_xyz = (nx, ny, nz)
    out = []
    for c in lat.C:
        blocked = torch.zeros(shape, dtype=torch.bool)
        for a in range(3):
            if not periodic[a] and c[a] != 0:
                src = coord_xyz[a] - c[a]
                blocked |= (src < 0) | (src >= extent_xyz[a])
        if solid is not None:
            blocked |= torch.roll(solid, shifts=(c[2], c[1], c[0]), dims=(0, 1, 2))
        out.append(blocked)
    return out


def stream(M, periodic, solid=None, mode="hermite", blocked=None):
    """Pull streaming with half-way bounce-back: returns f*[27, nz, ny, nx]."""
    fpost = lat.reconstruct(M, mode)
    if blocked is None:
        blocked = blocked_sources(tuple(M.shape[1:]), periodic, solid)
    fstar = torch.empty_like(fpost)
    for i, c in enumerate(lat.C):
        pulled = torch.roll(fpost[i], shifts=(c[2], c[1], c[0]), dims=(0, 1, 2))
        fstar[i] = torch.where(blocked[i], fpost[lat.OPP[i]], pulled)
    return fstar


def collide(fstar, tau, force=None, eps=None):
    """Moment-space collision (Sec. 3.1; mixture tau of Sec. 4; Guo forcing).

    Returns the post-collision stored moments M'[10, ...] and the physical
    velocity u (for diagnostics).
    """
    rho, j, Pi = lat.project(fstar)
    shape = tuple(rho.shape)
    F = _as_components(force, shape, fstar.dtype)
    u = [(j[a] + 0.5 * F[a]) / rho for a in range(3)]
    tau_e = tau if eps is None else eps * tau
    om = 1.0 / tau_e
    S = [[((1.0 - om) * Pi[a][b] + om * rho * u[a] * u[b]
           + (1.0 - 0.5 * om) * (u[a] * F[b] + F[a] * u[b])) / rho
          for b in range(3)] for a in range(3)]
    u_store = [u[a] + 0.5 * F[a] / rho for a in range(3)]
    return lat.pack_moments(rho, u_store, S), u


def step(M, tau, force=None, eps=None, periodic=(True, True, True), solid=None,
         mode="hermite", update=None, blocked=None):
    """One stream-collide step.  Nodes outside ``update`` (if given) and solid
    nodes keep their input moments."""
    fstar = stream(M, periodic, solid, mode, blocked)
    Mn, _ = collide(fstar, tau, force, eps)
    keep = torch.zeros(tuple(M.shape[1:]), dtype=torch.bool)
    if solid is not None:
        keep |= solid
    if update is not None:
        keep |= ~update
    return torch.where(keep.unsqueeze(0), M, Mn)


def run_open(M, n_steps, tau, types, inlet=(0.0, 0.0, 0.0, 1), force=None, eps=None, periodic=(True, True, True),
             solid=None, mode="hermite"):
    """Steps with open faces (``oracle.boundary``): the face layers keep their
    moments in the step and are then written from the state before it."""
    from . import boundary as bd
    shape = tuple(M.shape[1:])
    keep_open = bd.layer(shape, types)
    blocked = blocked_sources(shape, periodic, solid)
    for _ in range(n_steps):
        Mn = step(M, tau, force=force, eps=eps, periodic=periodic, solid=solid, mode=mode, update=~keep_open,
                  blocked=blocked)
        M = bd.apply(M, Mn, types, 0, inlet)
    return M


def run(M, n_steps, tau, **kw):
    """Apply ``step`` n times."""
    periodic = kw.get("periodic", (True, True, True))
    blocked = blocked_sources(tuple(M.shape[1:]), periodic, kw.get("solid"))
    for _ in range(n_steps):
        M = step(M, tau, blocked=blocked, **kw)
    return M


def physical_velocity(M, force=None):
    """u = u' - F/(2 rho): the velocity of Eq. (rho_u_stress) for stored moments M."""
    shape = tuple(M.shape[1:])
    F = _as_components(force, shape, M.dtype)
    return [M[1 + a] - 0.5 * F[a] / M[0] for a in range(3)]


def kinetic_energy(M, force=None, solid=None):
    """sum over fluid nodes of rho |u|^2 / 2 with the physical velocity."""
    u = physical_velocity(M, force)
    ke = 0.5 * M[0] * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    if solid is not None:
        ke = torch.where(solid, torch.zeros_like(ke), ke)
    return ke.sum()
