"""Pins for the oracle's open faces (convective outflow, logarithmic inlet).

* a uniform flow through a box with outflow faces on both ends of its axis
  stays uniform to rounding (the upwind update of an equal pair is the
  identity; the upstream face sees backflow and keeps its value);
* after one step the inlet layer holds, node by node, the density of its
  inward neighbour and u0 ln(1 + beta (h - h0)) along the inward normal on
  the profile axis (zero below h0), S = u u, on either side of the axis;
* the outflow layer moves towards its inward neighbour by the Courant number
  of that neighbour's outward velocity, and does not move under backflow;
* the multi-level driver with open faces reads no unstored node (the NaN fill
  stays out of every stored value).
"""
import math

import numpy as np
import pytest
import torch

from oracle import boundary as bd
from oracle import hierarchy as hy
from oracle import multilevel as ml
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

OUT2 = [bd.OUTFLOW, bd.OUTFLOW, 0, 0, 0, 0]


def uniform(shape, u):
    ux, uy, uz = (np.full(shape, v) for v in u)
    return torch.tensor(wl.equilibrium_field(np.ones(shape), ux, uy, uz))


def test_uniform_flow_passes_through_outflow_faces():
    shape = (8, 8, 16)
    M0 = uniform(shape, (0.03, 0.01, -0.02))
    M = sl.run_open(M0, 10, 0.8, OUT2, periodic=(False, True, True))
    assert (M - M0).abs().max() < 1e-14


def test_inlet_layer_holds_the_log_profile():
    shape = (8, 16, 16)  # z, y, x
    M0 = torch.tensor(wl.random_field(shape, 12, du=0.02))
    u0, beta, h0 = 0.05, 0.3, 2.5
    for side in (0, 1):
        types = [0] * 6
        types[side] = bd.INLET
        M1 = sl.run_open(M0, 1, 0.8, types, inlet=(u0, beta, h0, 1), periodic=(False, True, True))
        x = 0 if side == 0 else 15
        xi = 1 if side == 0 else 14
        sign = 1.0 if side == 0 else -1.0
        for y in range(16):
            arg = 1.0 + beta * (y - h0)
            u = u0 * math.log(arg) if arg > 1.0 else 0.0
            assert torch.allclose(M1[1, :, y, x], torch.full((8,), sign * u), atol=1e-15, rtol=0)
            assert torch.allclose(M1[4, :, y, x], torch.full((8,), u * u), atol=1e-15, rtol=0)
            assert M1[2:4, :, y, x].abs().max() == 0.0 and M1[5:, :, y, x].abs().max() == 0.0
            assert torch.equal(M1[0, :, y, x], M0[0, :, y, xi])


def test_outflow_layer_upwind_and_backflow():
    shape = (8, 8, 16)
    M0 = torch.tensor(wl.random_field(shape, 13, du=0.02))
    M0[1] = 0.05 + 0.02 * M0[1]          # flow towards +x everywhere
    M1 = sl.run_open(M0, 1, 0.8, OUT2, periodic=(False, True, True))
    c = M0[1, :, :, 14]                  # Courant number at the x+ face
    want = M0[:, :, :, 15] - c * (M0[:, :, :, 15] - M0[:, :, :, 14])
    assert torch.allclose(M1[:, :, :, 15], want, atol=1e-16, rtol=1e-14)
    assert torch.equal(M1[:, :, :, 0], M0[:, :, :, 0])   # backflow at the x- face


def test_multilevel_open_faces_read_no_unstored_node():
    ext = (16, 128, 16)
    O0 = np.zeros(hy.block_dims(ext, 8, 0), bool)
    O0[:, 7:9, :] = True
    h = hy.Hierarchy(O0, ext, 8, 2, (False, True, True))
    types = [bd.INLET, bd.OUTFLOW, 0, 0, 0, 0]
    m = ml.MultiLevel(h, 0.8, open_faces=(types, (0.04, 0.2, 4.0, 1)))
    for l in range(2):
        X, Y, Z = m.node_positions(l)
        ux = 0.02 + 0.01 * np.sin(2 * np.pi * Y / 128)
        m.set_level(l, wl.equilibrium_field(np.ones_like(ux), ux, 0 * ux, 0 * ux))
    for _ in range(3):
        m.coarse_step()
    for l in range(2):
        st = m.stored[l]
        assert torch.isfinite(m.current(l)[:, st]).all()
        assert torch.isnan(m.current(l)[:, ~st]).all() if (~st).any() else True
