"""Open faces (convective outflow, logarithmic inlet) on the GPU against the
oracle.

* single level, inlet on x- (profile along y), outflow on x+, walls on y:
  FP32 within 1e-5 per step of the row scale, FP16-scaled storage within its
  per-step bound; faces set after the blocks (neighbour tables rebuilt);
* two levels (a refined band across the open axis), faces set before the
  blocks: every level against the oracle's Algorithm 1 with the same faces;
* a uniform flow through outflow faces at both ends stays uniform;
* argument checks, and the adjoint is refused while a face is open.
"""
import numpy as np
import pytest
import torch

from oracle import boundary as bd
from oracle import hierarchy as hy
from oracle import multilevel as ml
from oracle import single_level as sl
from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl
from tests.helpers import rel_err, row_scales

pytestmark = pytest.mark.gpu

RP_TOL = {"f32": 1e-5, "f16s": 8 * 2.0 ** -11}
TYPES = [hl.FACE_INLET, hl.FACE_OUTFLOW, 0, 0, 0, 0]
INLET = (0.04, 0.3, 1.5, 1)


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_single_level_open_faces_match_oracle(storage):
    ext = (32, 16, 16)
    shape = (16, 16, 32)
    per = (False, False, True)
    M0 = wl.random_field(shape, 41, du=0.01)
    M0[1] += 0.03
    M0[4] = M0[1] * M0[1]
    steps = 8
    with hl.Lattice(ext, tau=0.8, periodic=per, storage=storage) as lat:
        lat.set_dense()
        lat.set_open_faces(TYPES, *INLET)
        lat.write_moments(hl.dense_to_blocks(M0))
        start = hl.blocks_to_dense(lat.read_moments(), shape)
        lat.step(steps)
        got = hl.blocks_to_dense(lat.read_moments(), shape)
    ref = sl.run_open(torch.tensor(start), steps, 0.8, TYPES, inlet=INLET, periodic=per).numpy()
    assert np.abs(ref[1, :, :, 0]).max() > 0.04      # the inlet profile is in place
    err = rel_err(got, ref, row_scales(ref, 0.03))
    assert err.max() < steps * RP_TOL[storage], err


def test_faces_changed_between_steps():
    """Faces changed after steps have run: the neighbour tables and the lists
    of open blocks are made again, and the next steps follow the oracle with
    the new faces (outflow at both x ends first, then inlet / outflow)."""
    ext = (32, 16, 16)
    shape = (16, 16, 32)
    per = (False, False, True)
    M0 = wl.random_field(shape, 43, du=0.01)
    M0[1] += 0.03
    M0[4] = M0[1] * M0[1]
    with hl.Lattice(ext, tau=0.8, periodic=per, storage="f32") as lat:
        lat.set_dense()
        lat.set_open_faces([hl.FACE_OUTFLOW, hl.FACE_OUTFLOW, 0, 0, 0, 0])
        lat.write_moments(hl.dense_to_blocks(M0))
        lat.step(3)
        lat.set_open_faces(TYPES, *INLET)
        start = hl.blocks_to_dense(lat.read_moments(), shape)
        lat.step(4)
        got = hl.blocks_to_dense(lat.read_moments(), shape)
    ref = sl.run_open(torch.tensor(start), 4, 0.8, TYPES, inlet=INLET, periodic=per).numpy()
    assert np.abs(ref[1, :, :, 0]).max() > 0.04
    err = rel_err(got, ref, row_scales(ref, 0.03))
    assert err.max() < 4 * RP_TOL["f32"], err


def test_two_level_open_faces_match_oracle():
    ext = (16, 128, 16)
    L = 2
    per = (False, True, True)
    O0 = np.zeros(hy.block_dims(ext, 8, 0), bool)
    O0[:, 7:9, :] = True
    h = hy.Hierarchy(O0, ext, 8, L, per)
    m0 = ml.MultiLevel(h, 0.8)
    lat = hl.Lattice(ext, levels=L, tau=0.8, periodic=per, storage="f32")
    with lat:
        lat.set_open_faces(TYPES, *INLET)
        z, y, x = np.nonzero(O0)
        lat.set_fine_blocks(np.stack([x, y, z], axis=1))
        coords = [lat.blocks(l)[0] for l in range(L)]
        for l in range(L):
            X, Y, Z = m0.node_positions(l)
            ux = 0.02 + 0.01 * np.sin(2 * np.pi * Y / 128)
            M = wl.equilibrium_field(np.ones_like(ux) + 1e-3 * np.cos(2 * np.pi * Z / 16), ux, 0.3 * ux,
                                     np.zeros_like(ux))
            lat.write_moments(hl.dense_to_blocks(M, coords[l]), level=l)
        m = ml.MultiLevel(h, 0.8, open_faces=(TYPES, INLET))
        for l in range(L):
            m.set_level(l, hl.blocks_to_dense(lat.read_moments(level=l), m.shape[l], coords[l]))
        for k in range(3):
            m.coarse_step()
            lat.step(2)
            for l in range(L):
                got = hl.blocks_to_dense(lat.read_moments(level=l), m.shape[l], coords[l])
                ref = m.current(l).numpy()
                err = rel_err(got, ref, row_scales(ref, 0.02), mask=m.stored[l].numpy())
                assert err.max() < 2e-5 * (k + 1), (k, l, err)


def test_uniform_flow_through_outflow_faces():
    shape = (16, 16, 32)
    ux, uy, uz = (np.full(shape, v) for v in (0.03, 0.01, -0.02))
    M0 = wl.equilibrium_field(np.ones(shape), ux, uy, uz)
    with hl.Lattice((32, 16, 16), tau=0.8, periodic=(False, True, True), storage="f32") as lat:
        lat.set_dense()
        lat.set_open_faces([hl.FACE_OUTFLOW, hl.FACE_OUTFLOW, 0, 0, 0, 0])
        lat.write_moments(hl.dense_to_blocks(M0))
        start = hl.blocks_to_dense(lat.read_moments(), shape)
        lat.step(10)
        got = hl.blocks_to_dense(lat.read_moments(), shape)
    assert np.abs(got - start).max() < 1e-6


def test_open_face_arguments_and_adjoint_refusal():
    with hl.Lattice((32, 16, 16), tau=0.8, periodic=(False, True, True), storage="f32") as lat:
        lat.set_dense()
        with pytest.raises(hl.HlbmError) as ei:   # y is periodic
            lat.set_open_faces([0, 0, hl.FACE_OUTFLOW, 0, 0, 0])
        assert ei.value.code == hl.E_INVALID_ARG
        with pytest.raises(hl.HlbmError) as ei:   # profile axis across the inlet face
            lat.set_open_faces(TYPES, 0.04, 0.3, 1.5, 0)
        assert ei.value.code == hl.E_INVALID_ARG
        with pytest.raises(hl.HlbmError) as ei:
            lat.set_open_faces([7, 0, 0, 0, 0, 0])
        assert ei.value.code == hl.E_INVALID_ARG
        lat.set_open_faces(TYPES, *INLET)
        with pytest.raises(hl.HlbmError) as ei:
            lat.forward_record(4, 2)
        assert ei.value.code == hl.E_UNSUPPORTED
        lat.set_open_faces([0] * 6)
        lat.forward_record(4, 2)
