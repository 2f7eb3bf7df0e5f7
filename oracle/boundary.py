"""Open faces of the domain: convective outflow and logarithmic inlet.

Test infrastructure (see ``oracle/__init__.py``).  Sec. 7 (dune and ripple
scenes): at an outlet the boundary cells solve dM/dt + u_n dM/dn = 0 with
u_n the fluid speed of the nearest interior neighbour along the boundary
normal; the ripple scene drives the wind with u_x(y) = u_0 ln(1 + beta (y -
y_0)) at the inlet.  Readings of what the paper leaves open:

* the face layer is the outermost node layer; it keeps its moments in the
  level step and is then written from the state before the step;
* outflow: first-order upwind in time and space with unit steps,
  M_b <- M_b - c (M_b - M_i), c = clamp(u_n, 0, 1), M_i the node one step
  inward, u_n its stored velocity along the outward normal (no backflow);
* inlet: density of M_i, velocity u(h) along the inward normal, zero where
  1 + beta (h - h0) <= 1, S = u u; h is the node's coordinate along the
  profile axis in finest-level node units (level-l node i sits at i 2^l);
* a node on several open faces takes the first of x-, x+, y-, y+, z-, z+.

Faces are numbered f = 2 axis + side (axis x = 0, y = 1, z = 2; side 0 = low).
Types: 0 closed, 1 outflow, 2 inlet.  Arrays are indexed [z, y, x].
"""
import math

import torch

CLOSED, OUTFLOW, INLET = 0, 1, 2


def _dim(axis):
    """Array dimension (of a (nz, ny, nx) grid) holding coordinate ``axis``."""
    return 2 - axis


def face_masks(shape, types):
    """For each face f, the bool mask of the nodes it writes (first open face wins)."""
    taken = torch.zeros(shape, dtype=torch.bool)
    out = []
    for f in range(6):
        m = torch.zeros(shape, dtype=torch.bool)
        if types[f] != CLOSED:
            d = _dim(f >> 1)
            idx = [slice(None)] * 3
            idx[d] = 0 if (f & 1) == 0 else shape[d] - 1
            m[tuple(idx)] = True
            m &= ~taken
            taken |= m
        out.append(m)
    return out


def layer(shape, types):
    """All nodes of the open face layers."""
    ms = face_masks(shape, types)
    out = torch.zeros(shape, dtype=torch.bool)
    for m in ms:
        out |= m
    return out


def apply(M_old, M_new, types, level=0, inlet=(0.0, 0.0, 0.0, 1), stored=None):
    """Write the open-face nodes of M_new (10, nz, ny, nx) from M_old (only
    those in ``stored`` if given: the others keep their value)."""
    u0, beta, h0, paxis = inlet
    shape = tuple(M_old.shape[1:])
    out = M_new.clone()
    for f, m in enumerate(face_masks(shape, types)):
        if stored is not None:
            m = m & stored
        if types[f] == CLOSED or not bool(m.any()):
            continue
        axis, hi = f >> 1, f & 1
        d = _dim(axis)
        inward = -1 if hi else 1
        Mi = torch.roll(M_old, shifts=-inward, dims=1 + d)  # value of the node one step inward
        if types[f] == OUTFLOW:
            un = Mi[1 + axis] if hi else -Mi[1 + axis]
            c = torch.clamp(un, 0.0, 1.0)
            val = M_old - c.unsqueeze(0) * (M_old - Mi)
        else:
            n = shape[_dim(paxis)]
            hcoord = torch.arange(n, dtype=M_old.dtype) * float(2 ** level)
            arg = 1.0 + beta * (hcoord - h0)
            prof = torch.where(arg > 1.0, u0 * torch.log(torch.clamp(arg, min=1.0)), torch.zeros_like(arg))
            view = [1, 1, 1]
            view[_dim(paxis)] = n
            u = prof.reshape(view).expand(shape) * float(inward)
            uv = [torch.zeros(shape, dtype=M_old.dtype) for _ in range(3)]
            uv[axis] = u
            val = torch.stack([Mi[0], uv[0], uv[1], uv[2], uv[0] * uv[0], uv[1] * uv[1], uv[2] * uv[2],
                               uv[0] * uv[1], uv[0] * uv[2], uv[1] * uv[2]])
        out = torch.where(m.unsqueeze(0), val, out)
    return out
