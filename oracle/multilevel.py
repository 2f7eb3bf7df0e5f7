"""Multi-level advance of Algorithm 1 with downward/upward transfers.

Test infrastructure (see ``oracle/__init__.py``).  Every level is held as a
dense FP64 array at that level's node resolution (nodes of level l sit at fine
positions 2^l * index: vertex-aligned levels, Sec. 5.1 "one block shift" and
Sec. 5.3 "corresponding node"); nodes that are not stored hold NaN so that any
read of them poisons the result.  Each level has two buffers and reads the one
selected by its own step parity, which is the two-tree recursive ping-pong of
Sec. 6.2 written per level.

Passages followed:
* tau_{l+1} = tau_l / 2 + 1/4 (Sec. 5.2, the nu/tau rescaling with k = 1);
* Algorithm 1 AdvanceLBM(l, s): DownwardTransfer(l+1, s) before the level-l
  step, UpwardTransfer(l) after it when s = 2, then two sub-steps of level l-1;
* DownwardTransfer: rho and u interpolated over the 2^D nearest coarse nodes,
  S = k_down sum_j w_j S^neq_j + S^eq with S^eq = u u from the interpolated u;
  at s = 2 the coarse state is the temporal midpoint of the old and new coarse
  states (Eq. downward_rescale and the paragraph after it);
* UpwardTransfer: copy rho, u of the coincident fine node, S = k_up S^neq + S^eq
  (Eq. upload_S).

The S^neq scale factors of the paper are not inverse to each other; the
``rescale`` argument selects a reading (see ``rescale_factors``).
"""
import numpy as np
import torch

from . import boundary as bd
from . import coupling as cp
from . import lattice as lat
from . import single_level as sl


def level_taus(tau0, L):
    """tau_{l+1} = tau_l/2 + 1/4 (Sec. 5.2 with k = 1)."""
    t = [float(tau0)]
    for _ in range(1, L):
        t.append(t[-1] / 2.0 + 0.25)
    return t


def rescale_factors(tau_f, tau_c, rescale):
    """(k_up, k_down) for S^neq between a fine level (tau_f) and the next coarser one (tau_c).

    * ``post``  : S^neq of the stored (post-collision) moments scales with
                  (tau - 1) times the lattice velocity gradient, which doubles per
                  level: k_up = 2 (tau_c - 1)/(tau_f - 1), k_down = 1/k_up;
    * ``pre``   : Chapman-Enskog scaling of the pre-collision S^neq with tau:
                  k_up = 2 tau_c / tau_f, k_down = 1/k_up;
    * ``paper`` : the factors as printed, k_up = tau_c/(2 tau_f) (Eq. upload_S),
                  k_down = 2 tau_c / tau_f (Eq. downward_rescale).
    """
    if rescale == "post":
        k = 2.0 * (tau_c - 1.0) / (tau_f - 1.0)
        return k, 1.0 / k
    if rescale == "pre":
        k = 2.0 * tau_c / tau_f
        return k, 1.0 / k
    if rescale == "paper":
        return tau_c / (2.0 * tau_f), 2.0 * tau_c / tau_f
    raise ValueError(rescale)


def split_neq(M):
    """(rho, u[3], S^neq[6]) with S^neq = S - u u in the stored row order."""
    rho, ux, uy, uz = M[0], M[1], M[2], M[3]
    eq = [ux * ux, uy * uy, uz * uz, ux * uy, ux * uz, uy * uz]
    return rho, [ux, uy, uz], [M[4 + r] - eq[r] for r in range(6)]


def join_neq(rho, u, sneq, k):
    """Stored moments from rho, u and k * S^neq + u u."""
    ux, uy, uz = u
    eq = [ux * ux, uy * uy, uz * uz, ux * uy, ux * uz, uy * uz]
    return torch.stack([rho, ux, uy, uz] + [k * sneq[r] + eq[r] for r in range(6)])


def _axis_pair(p, n_coarse, periodic):
    """Coarse indices (floor(p/2), ceil(p/2)) along one axis; ceil wraps on a
    periodic axis and is clamped to the last coarse node on a wall axis."""
    lo = p // 2
    hi = (p + 1) // 2
    if periodic:
        hi = hi % n_coarse
    else:
        hi = np.minimum(hi, n_coarse - 1)
    return lo, hi


def interpolate_down(Mc, nodes, periodic, k_down):
    """Spatial part of Eq. (downward_rescale) at fine nodes ``nodes`` = (pz, py, px).

    Each axis contributes the coarse nodes floor(p/2) and ceil(p/2) with weight
    1/2 each (for even p both are the coincident node), i.e. trilinear weights
    over the 2^D nearest coarse nodes.  Mc is (rho, u[3], S^neq[6]) of the
    coarse level.  Returns stored moments (10, n_nodes).
    """
    pz, py, px = nodes
    ncz, ncy, ncx = Mc[0].shape
    zs = _axis_pair(pz, ncz, periodic[2])
    ys = _axis_pair(py, ncy, periodic[1])
    xs = _axis_pair(px, ncx, periodic[0])
    rho_c, u_c, s_c = Mc
    rho = 0.0
    u = [0.0, 0.0, 0.0]
    s = [0.0] * 6
    for cz in zs:
        for cy in ys:
            for cx in xs:
                idx = (torch.as_tensor(cz), torch.as_tensor(cy), torch.as_tensor(cx))
                rho = rho + 0.125 * rho_c[idx]
                for a in range(3):
                    u[a] = u[a] + 0.125 * u_c[a][idx]
                for r in range(6):
                    s[r] = s[r] + 0.125 * s_c[r][idx]
    return join_neq(rho, u, s, k_down)


class MultiLevel:
    """State and Algorithm 1 driver over a fixed ``oracle.hierarchy.Hierarchy``."""

    def __init__(self, hier, tau0, mode="hermite", rescale="post", force=None, eps=None, drag=None, open_faces=None):
        self.h = hier
        self.L = hier.L
        self.mode = mode
        self.rescale = rescale
        self.tau = level_taus(tau0, self.L)
        self.force = force          # level-0 dense (3, nz, ny, nx) tensor, tuple or None
        self.eps = eps              # level-0 dense (nz, ny, nx) tensor or None
        self.drag = drag            # (kappa, vp, every): coupled level-0 steps (``coupling``)
        self.open_faces = open_faces  # (types[6], (u0, beta, h0, axis)): open faces (``boundary``)
        self.l0_steps = 0
        self.periodic = hier.periodic
        self.buf = [[None, None] for _ in range(self.L)]
        self.cur = [0] * self.L
        self._masks()

    def _masks(self):
        h = self.h
        self.shape = []
        self.update, self.down, self.up, self.stored, self.blocked = [], [], [], [], []
        for l in range(self.L):
            st = h.stored_nodes(l)
            miss = h.missing_nodes(l)
            self.shape.append(st.shape)
            self.stored.append(torch.as_tensor(st))
            upd = torch.as_tensor(st & ~miss)
            if self.open_faces is not None:
                upd &= ~bd.layer(tuple(st.shape), self.open_faces[0])
            self.update.append(upd)
            self.down.append(np.nonzero(h.down_nodes(l)))
            self.up.append(np.nonzero(h.up_nodes(l)))
            self.blocked.append(sl.blocked_sources(st.shape, self.periodic))

    # ---------------------------------------------------------------- state
    def node_positions(self, l):
        """Fine-unit positions (x, y, z) of every level-l node, each (nz_l, ny_l, nx_l)."""
        nz, ny, nx = self.shape[l]
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        s = float(1 << l)
        return x * s, y * s, z * s

    def set_level(self, l, M, fill=None, dtype=torch.float64):
        """Set both buffers of level l from a dense (10, nz_l, ny_l, nx_l) array.

        Nodes that are not stored become NaN, so that any read of them poisons
        the result; ``fill`` (10 values) puts a finite state there instead,
        for reverse-mode differentiation, where 0 * NaN in the chain rule
        would poison gradients that do not depend on those nodes."""
        M = torch.as_tensor(M).to(dtype).clone()
        if fill is None:
            M[:, ~self.stored[l]] = float("nan")
        else:
            M[:, ~self.stored[l]] = torch.as_tensor(fill, dtype=dtype).unsqueeze(1)
        self.buf[l] = [M.clone(), M.clone()]
        self.cur[l] = 0

    def current(self, l):
        return self.buf[l][self.cur[l]]

    def previous(self, l):
        return self.buf[l][1 - self.cur[l]]

    def k_updown(self, l):
        """(k_up, k_down) between level l and level l+1."""
        return rescale_factors(self.tau[l], self.tau[l + 1], self.rescale)

    # ---------------------------------------------------------------- Algorithm 1
    def streaming_collision(self, l):
        M = self.current(l)
        force = self.force if l == 0 else None
        eps = self.eps if l == 0 else None
        if l == 0 and self.drag is not None and self.l0_steps % self.drag[2] == 0:
            # S, drag exchange, C (Fig. 4); the drag is the level-0 force until the next exchange
            Mn, self.force = cp.coupled_step(M, self.tau[0], eps, self.drag[1], self.drag[0],
                                             periodic=self.periodic, mode=self.mode,
                                             update=self.update[0], blocked=self.blocked[0])
        else:
            Mn = sl.step(M, self.tau[l], force=force, eps=eps, periodic=self.periodic,
                         mode=self.mode, update=self.update[l], blocked=self.blocked[l])
        if self.open_faces is not None:
            Mn = bd.apply(M, Mn, self.open_faces[0], l, self.open_faces[1], stored=self.stored[l])
        if l == 0:
            self.l0_steps += 1
        self.buf[l][1 - self.cur[l]] = Mn
        self.cur[l] = 1 - self.cur[l]

    def downward_transfer(self, lc, s):
        """DownwardTransfer(l+1, s): fill I^d_l of level l = lc-1 (its read buffer)."""
        l = lc - 1
        nodes = self.down[l]
        if len(nodes[0]) == 0:
            return
        old = split_neq(self.previous(lc))
        if s == 1:
            Mc = old
        else:
            new = split_neq(self.current(lc))
            Mc = (0.5 * (old[0] + new[0]),
                  [0.5 * (old[1][a] + new[1][a]) for a in range(3)],
                  [0.5 * (old[2][r] + new[2][r]) for r in range(6)])
        _, k_down = self.k_updown(l)
        vals = interpolate_down(Mc, nodes, self.periodic, k_down)
        self._assign(l, nodes, vals)

    def _assign(self, l, nodes, vals):
        """Overwrite ``nodes`` of level l's read buffer.  The buffer is replaced
        by an updated copy rather than written in place, so that reverse-mode
        differentiation can still use the values earlier operations read."""
        M = self.current(l).clone()
        M[:, nodes[0], nodes[1], nodes[2]] = vals
        self.buf[l][self.cur[l]] = M

    def upward_transfer(self, l):
        """UpwardTransfer(l): I^u_{l+1} nodes copy their coincident level-l node (Eq. upload_S)."""
        nodes = self.up[l + 1]
        if len(nodes[0]) == 0:
            return
        k_up, _ = self.k_updown(l)
        Mf = self.current(l)
        fz, fy, fx = (2 * nodes[0], 2 * nodes[1], 2 * nodes[2])
        rho, u, sneq = split_neq(Mf[:, fz, fy, fx])
        self._assign(l + 1, nodes, join_neq(rho, u, sneq, k_up))

    def advance(self, l, s):
        """AdvanceLBM(l, s) of Algorithm 1."""
        if l < self.L - 1:
            self.downward_transfer(l + 1, s)
        self.streaming_collision(l)
        if l < self.L - 1 and s == 2:
            self.upward_transfer(l)
        if l > 0:
            self.advance(l - 1, 1)
            self.advance(l - 1, 2)

    def coarse_step(self):
        """One top-level call: 2^(L-1) fine steps."""
        self.advance(self.L - 1, 1)

    # ---------------------------------------------------------------- rebuild
    def refresh_down_nodes(self):
        """At a coarse-step boundary every level is at the same time: refill each
        I^d_l from the current state of level l+1 (spatial rule only), top-down."""
        for l in range(self.L - 2, -1, -1):
            nodes = self.down[l]
            if len(nodes[0]) == 0:
                continue
            _, k_down = self.k_updown(l)
            self.current(l)[:, nodes[0], nodes[1], nodes[2]] = interpolate_down(
                split_neq(self.current(l + 1)), nodes, self.periodic, k_down)

    def complete_fields(self):
        """Per-level dense fields where every node that any level can supply is filled.

        Stored nodes keep their value.  Then, bottom-up, a node missing at level
        l takes the upward rule from the coincident node of level l-1; then,
        top-down, a node still missing takes the downward spatial rule from level
        l+1 if all its coarse stencil nodes are known.
        """
        fill = [self.current(l).clone() for l in range(self.L)]
        for l in range(1, self.L):
            k_up, _ = self.k_updown(l - 1)
            nz, ny, nx = self.shape[l]
            sub = fill[l - 1][:, 0::2, 0::2, 0::2][:, :nz, :ny, :nx]
            rho, u, sneq = split_neq(sub)
            cand = join_neq(rho, u, sneq, k_up)
            need = torch.isnan(fill[l][0]) & ~torch.isnan(cand[0])
            fill[l] = torch.where(need.unsqueeze(0), cand, fill[l])
        for l in range(self.L - 2, -1, -1):
            miss = torch.isnan(fill[l][0]).numpy()
            nodes = np.nonzero(miss)
            if len(nodes[0]) == 0:
                continue
            _, k_down = self.k_updown(l)
            vals = interpolate_down(split_neq(fill[l + 1]), nodes, self.periodic, k_down)
            fill[l][:, nodes[0], nodes[1], nodes[2]] = vals
        return fill

    def rebuild(self, new_hier):
        """Switch to ``new_hier`` at a coarse-step boundary (Sec. 6.3): surviving
        nodes keep their moments, new fine nodes are interpolated from their
        parents (Eq. downward_rescale, spatial part), new coarse nodes take the
        upward rule from their children (Eq. upload_S)."""
        self.refresh_down_nodes()
        fill = self.complete_fields()
        old = self.h
        self.h = new_hier
        self._masks()
        for l in range(self.L):
            M = fill[l].clone()
            M[:, ~self.stored[l]] = float("nan")
            if torch.isnan(M[:, self.stored[l]]).any():
                raise RuntimeError("rebuild: a new node has no source at any level")
            self.buf[l] = [M.clone(), M.clone()]
            self.cur[l] = 0
        return old

    # ---------------------------------------------------------------- reductions
    def reduce(self):
        """FP64 mass, momentum (3), kinetic energy over owned nodes, cell volume 8^l.

        Returns [mass, px, py, pz, ke, mass_level0, mass_other_levels] with the
        physical velocity at level 0 (force shift removed).
        """
        out = np.zeros(7)
        for l in range(self.L):
            M = self.current(l)
            own = torch.as_tensor(self.h.owned_nodes(l))
            vol = float(8 ** l)
            force = self.force if l == 0 else None
            u = sl.physical_velocity(M, force)
            rho = M[0]
            m = (rho[own].sum() * vol).item()
            out[0] += m
            for a in range(3):
                out[1 + a] += (rho * u[a])[own].sum().item() * vol
            out[4] += (0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))[own].sum().item() * vol
            if l == 0:
                out[5] += m
            else:
                out[6] += m
        return out
