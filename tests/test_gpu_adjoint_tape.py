"""The recording pass runs its last checkpoint segment the way the adjoint
recomputes one and keeps it (the tape); the first adjoint starts from the
tape, a second adjoint on the same recording recomputes every segment.

* both adjoints give bit-identical dL/dF (single level with a partial last
  segment, two and three levels);
* the state the recording leaves is bit for bit the state of plain steps;
* a recording refused for lack of memory keeps no tape (covered with the
  injected failures of test_gpu_oom.py).
"""
import numpy as np
import pytest
import torch

from paper_2603_14982_gb300 import homelbm as hl
from paper_2603_14982_gb300 import workloads as wl
from tests.helpers import ml_adjoint_case

pytestmark = pytest.mark.gpu


def _single_level(extent=(32, 16, 16)):
    nx, ny, nz = extent
    shape = (nz, ny, nx)
    lat = hl.Lattice(extent, tau=0.7, periodic=(True, False, False), storage="f32")
    lat.set_dense()
    solid = np.zeros(shape, dtype=np.uint8)
    solid[6:10, 6:10, 12:16] = 1
    lat.set_solid(solid)
    lat.write_moments(hl.dense_to_blocks(wl.random_field(shape, 71, du=0.02, drho=1e-3, dneq=1e-4)))
    F = wl.noisy_force(shape, seed=72, mean=(1e-5, 0.0, 0.0), sigma=1e-5)
    lat.set_force(torch.tensor(hl.dense_to_blocks(F), dtype=torch.float32, device="cuda"))
    return lat, [lat.blocks(0)[0]]


def _multi_level(name):
    c = ml_adjoint_case(name)
    lat = hl.Lattice(c["ext"], levels=c["L"], tau=c["tau0"], periodic=c["periodic"], storage="f32")
    z, y, x = np.nonzero(c["O0"])
    lat.set_fine_blocks(np.stack([x, y, z], axis=1))
    coords = [lat.blocks(l)[0] for l in range(c["L"])]
    for l in range(c["L"]):
        lat.write_moments(hl.dense_to_blocks(c["M0"][l], coords[l]), level=l)
    lat.set_force(torch.tensor(hl.dense_to_blocks(c["F"].astype(np.float32), coords[0]), device="cuda"))
    return lat, coords


@pytest.mark.parametrize("case", ["single", "two_level", "three_level_wall"])
def test_taped_and_recomputed_adjoints_agree(case):
    if case == "single":
        lat, coords = _single_level()
        n_steps, ckpt = 12, 5          # segments of 5, 5 and 2 steps: the tape holds a partial one
    else:
        lat, coords = _multi_level(case)
        per = 1 << (len(coords) - 1)
        n_steps, ckpt = 3 * per, 2 * per
    L = len(coords)
    with lat:
        start = [lat.read_moments(level=l) for l in range(L)]
        lat.step(n_steps)
        plain = [lat.read_moments(level=l, dtype=np.float32) for l in range(L)]
        for l in range(L):
            lat.write_moments(start[l], level=l)
        lat.forward_record(n_steps, ckpt)
        recorded = [lat.read_moments(level=l, dtype=np.float32) for l in range(L)]
        for l in range(L):
            assert np.array_equal(recorded[l].view(np.uint32), plain[l].view(np.uint32)), l
        g = torch.Generator().manual_seed(5)
        W = torch.randn((sum(len(cl) for cl in coords), 10, 512), generator=g).cuda()
        d1 = torch.empty((len(coords[0]), 3, 512), dtype=torch.float32, device="cuda")
        d2 = torch.empty_like(d1)
        lat.adjoint(W, d1)   # from the tape
        lat.adjoint(W, d2)   # every segment recomputed
        a, b = d1.cpu().numpy(), d2.cpu().numpy()
        assert np.isfinite(a).all() and np.abs(a).max() > 0
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
