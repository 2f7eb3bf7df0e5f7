"""The interface transfers narrow their FP64 sums to FP32 with integer
arithmetic (round to nearest, ties to even, Sec. 5.2 transfers); this checks
that narrowing bit for bit against the CUDA conversion instruction on values
that probe every branch: random magnitudes across the binary32 range, exact
ties (half an ulp, odd and even), round-ups that carry into the exponent or
overflow to infinity, the binary32 subnormal range, signed zeros,
infinities and NaNs."""
import numpy as np
import pytest
import torch

from paper_2603_14982_gb300 import homelbm as hl

pytestmark = pytest.mark.gpu


def probe_values(seed=3):
    rng = np.random.default_rng(seed)
    v = [rng.standard_normal(200_000) * 10.0 ** rng.uniform(-40, 38, 200_000),
         rng.uniform(-1, 1, 100_000)]
    # exact ties and neighbours: a float32 value plus half an ulp (+- one double ulp)
    f = rng.standard_normal(50_000).astype(np.float32) * np.float32(2.0) ** rng.integers(-120, 120, 50_000)
    f = f[np.isfinite(f) & (f != 0)]
    with np.errstate(over="ignore"):
        half = np.spacing(np.abs(f)).astype(np.float64) / 2
    base = f.astype(np.float64)
    for d in (half, -half):
        t = base + np.sign(base) * d
        v += [t, np.nextafter(t, np.inf), np.nextafter(t, -np.inf)]
    top = np.float64(np.finfo(np.float32).max)  # its ulp is 2^104
    v.append(np.array([top, top + 2.0 ** 103, top + 2.0 ** 103 * (1 - 2 ** -40), -top * (1 + 2 ** -25),
                       2.0 ** 128, 2.0 ** -126, 2.0 ** -126 * (1 - 2 ** -40), 2.0 ** -127, 2.0 ** -149,
                       2.0 ** -150, 2.0 ** -151, 1.0 - 2 ** -25, 1.0 + 2 ** -24, 1.0 + 3 * 2 ** -24,
                       0.0, -0.0, np.inf, -np.inf, np.nan, 1e-300, -1e300]))
    return np.concatenate(v)


def test_narrowing_matches_conversion_instruction():
    x = probe_values()
    xin = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    hw = torch.empty_like(out)
    lib = hl.load()
    assert lib.hlbm_test_narrow(xin.data_ptr(), out.data_ptr(), hw.data_ptr(), x.size) == hl.OK
    a = out.cpu().numpy().view(np.uint32)
    b = hw.cpu().numpy().view(np.uint32)
    nan = np.isnan(out.cpu().numpy())
    assert np.array_equal(nan, np.isnan(hw.cpu().numpy()))
    assert np.array_equal(a[~nan], b[~nan])
    # the probes reach the rounding branches they are meant for
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)  # numpy rounds to nearest, ties to even
    assert np.array_equal(a[~nan], ref[~nan].view(np.uint32))


def test_narrowing_hook_arguments():
    lib = hl.load()
    assert lib.hlbm_test_narrow(None, None, None, 0) == hl.OK
    assert lib.hlbm_test_narrow(None, None, None, 5) == hl.E_INVALID_ARG
