"""Declarative multi-level block hierarchy (Sec. 5.1, Sec. 6.1, Sec. 6.3).

Test infrastructure (see ``oracle/__init__.py``).  Plain numpy on dense
boolean block grids, one per level, indexed [bz, by, bx].  Level l has block
edge B cells of spacing 2^l (fine units); level 0 is the finest.

Reading of the paper used here:
* the level-selection function Phi (Sec. 5.4) is 0 on a level-0 block holding a
  particle and L-1 elsewhere, so the occupied set O_0 drives everything;
* H_l = level-l blocks that have stored children: H_1 = dilate(parent(O_0)),
  H_l = dilate(parent(H_{l-1})), dilation by one block in the 26-neighbourhood
  (clipped at walls, wrapped on periodic axes) -- the overlap/separation of
  Sec. 5.3 and Sec. 6.1 with whole 8^3 blocks;
* internal blocks I_l = {b in H_l : every in-domain 26-neighbour is in H_l} are
  not stored (Sec. 6.1: only leaf and border tiles are stored);
* stored_l = children(H_{l+1}) minus I_l for l < L-1, all blocks minus I_{L-1}
  at the top level; a stored block is ``border`` if it overlaps the finer
  level (in H_l) or the coarser one (its parent is stored), else ``leaf``;
* the flags of Sec. 6.3 are set differences against the previous hierarchy:
  refine = newly in H_l, coarsen = newly out of H_l, delete = no longer stored.
"""
import numpy as np

LEAF, BORDER, NEW, REFINE, COARSEN = 1, 2, 4, 8, 16


def block_dims(extent_xyz, B, level):
    """(nbz, nby, nbx) of the level-l block grid for a fine-equivalent extent."""
    s = B * (1 << level)
    nx, ny, nz = extent_xyz
    assert nx % s == 0 and ny % s == 0 and nz % s == 0
    return (nz // s, ny // s, nx // s)


def _shift(G, d, axis, periodic, fill):
    """G shifted so that out[idx] = G[idx + d] along ``axis`` (numpy axis)."""
    if d == 0:
        return G
    if periodic:
        return np.roll(G, -d, axis=axis)
    out = np.full_like(G, fill)
    n = G.shape[axis]
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    if d > 0:
        src[axis] = slice(d, n)
        dst[axis] = slice(0, n - d)
    else:
        src[axis] = slice(0, n + d)
        dst[axis] = slice(-d, n)
    out[tuple(dst)] = G[tuple(src)]
    return out


def neighbour(G, dx, dy, dz, periodic, fill):
    """out[b] = G[b + (dx,dy,dz)]; out-of-domain (non-periodic) reads ``fill``."""
    px, py, pz = periodic
    out = _shift(G, dz, 0, pz, fill)
    out = _shift(out, dy, 1, py, fill)
    return _shift(out, dx, 2, px, fill)


OFFSETS26 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
             if (dx, dy, dz) != (0, 0, 0)]


def dilate(G, periodic):
    out = G.copy()
    for d in OFFSETS26:
        out |= neighbour(G, *d, periodic, False)
    return out


def parent(G):
    """Level-(l+1) grid: a block is set if any of its 2x2x2 children is set."""
    nz, ny, nx = G.shape
    return G.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).any(axis=(1, 3, 5))


def children(G):
    return G.repeat(2, 0).repeat(2, 1).repeat(2, 2)


def internal(H, periodic):
    out = H.copy()
    for d in OFFSETS26:
        out &= neighbour(H, *d, periodic, True)
    return out


def occupancy(pos, extent_xyz, B):
    """O_0: level-0 blocks holding at least one particle (Phi = 0 there, Sec. 5.4).

    ``pos`` is (n, 3) float32 in fine-cell units (x, y, z); the block of a
    particle is floor(p / B), clamped into the domain.
    """
    dims = block_dims(extent_xyz, B, 0)
    O = np.zeros(dims, dtype=bool)
    if len(pos) == 0:
        return O
    b = np.floor(np.asarray(pos, dtype=np.float32) / np.float32(B)).astype(np.int64)
    b[:, 0] = np.clip(b[:, 0], 0, dims[2] - 1)
    b[:, 1] = np.clip(b[:, 1], 0, dims[1] - 1)
    b[:, 2] = np.clip(b[:, 2], 0, dims[0] - 1)
    O[b[:, 2], b[:, 1], b[:, 0]] = True
    return O


class Hierarchy:
    """Block sets of every level for one occupancy O_0 (or, through ``from_H``,
    for given has-children sets H_l)."""

    def __init__(self, O0, extent_xyz, B, L, periodic, H=None):
        self.extent, self.B, self.L, self.periodic = tuple(extent_xyz), B, L, tuple(periodic)
        self.dims = [block_dims(extent_xyz, B, l) for l in range(L)]
        if H is None:
            H = [np.zeros(self.dims[0], dtype=bool)]
            if L > 1:
                H.append(dilate(parent(O0), periodic))
                for l in range(2, L):
                    H.append(dilate(parent(H[l - 1]), periodic))
        else:
            H = [np.asarray(g, dtype=bool) for g in H]
            O0 = np.zeros(self.dims[0], dtype=bool)
        I = [np.zeros(self.dims[0], dtype=bool)] + [internal(H[l], periodic) for l in range(1, L)]
        stored = []
        for l in range(L):
            if l < L - 1:
                stored.append(children(H[l + 1]) & ~I[l])
            else:
                stored.append(~I[l])
        border = []
        for l in range(L):
            b = stored[l] & H[l]
            if l < L - 1:
                b |= stored[l] & children(stored[l + 1])
            border.append(b)
        self.O0, self.H, self.I, self.stored, self.border = O0, H, I, stored, border

    @classmethod
    def from_H(cls, H, extent_xyz, B, L, periodic):
        """The hierarchy of given has-children sets H[l] (H[0] empty): a level
        can be refined in regions no finer level needs (a level-selection
        function Phi that takes intermediate levels, Sec. 5.4)."""
        return cls(None, extent_xyz, B, L, periodic, H=H)

    # ---- block lists in ascending linear slot id z*(nby*nbx) + y*nbx + x
    def blocks(self, l):
        """int32 (n, 3) coordinates (bx, by, bz) of stored level-l blocks, slot order."""
        z, y, x = np.nonzero(self.stored[l])          # C order == ascending slot id
        return np.stack([x, y, z], axis=1).astype(np.int32)

    def flags(self, l, prev=None):
        """uint8 flag per stored block (same order as ``blocks``)."""
        z, y, x = np.nonzero(self.stored[l])
        f = np.where(self.border[l][z, y, x], BORDER, LEAF).astype(np.uint8)
        if prev is not None:
            f |= np.where(~prev.stored[l][z, y, x], NEW, 0).astype(np.uint8)
            f |= np.where(self.H[l][z, y, x] & ~prev.H[l][z, y, x], REFINE, 0).astype(np.uint8)
            f |= np.where(~self.H[l][z, y, x] & prev.H[l][z, y, x], COARSEN, 0).astype(np.uint8)
        return f

    def counts(self, prev):
        """(refined, coarsened, deleted) block counts over all levels vs ``prev``."""
        ref = sum(int((self.H[l] & ~prev.H[l]).sum()) for l in range(self.L))
        coa = sum(int((~self.H[l] & prev.H[l]).sum()) for l in range(self.L))
        dele = sum(int((prev.stored[l] & ~self.stored[l]).sum()) for l in range(self.L))
        return ref, coa, dele

    # ---- node-level masks (dense arrays at level-l node resolution)
    def node_grid(self, G, l):
        B = self.B
        return G.repeat(B, 0).repeat(B, 1).repeat(B, 2)

    def stored_nodes(self, l):
        return self.node_grid(self.stored[l], l)

    def missing_nodes(self, l):
        """Stored level-l nodes with a 26-neighbour node that is not stored.

        Neighbours beyond a wall do not count (bounce-back handles them).
        """
        s = self.stored_nodes(l)
        miss = np.zeros_like(s)
        for d in OFFSETS26:
            miss |= ~neighbour(s, *d, self.periodic, True)
        return s & miss

    def up_nodes(self, l):
        """I^u_l: missing-neighbour nodes inside H_l (filled from level l-1)."""
        return self.missing_nodes(l) & self.node_grid(self.H[l], l)

    def down_nodes(self, l):
        """I^d_l: missing-neighbour nodes outside H_l (filled from level l+1)."""
        return self.missing_nodes(l) & ~self.node_grid(self.H[l], l)

    def owned_nodes(self, l):
        """Stored level-l nodes not covered by a finer level (for reductions)."""
        return self.stored_nodes(l) & ~self.node_grid(self.H[l], l)


def from_particles(pos, extent_xyz, B, L, periodic):
    return Hierarchy(occupancy(pos, extent_xyz, B), extent_xyz, B, L, periodic)
