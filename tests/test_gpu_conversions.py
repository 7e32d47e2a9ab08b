"""The integer-pipe float/double conversions of the downward and force passes
(and of the mixed precision's packing) against the GPU's own conversion
instructions, bit for bit, through the library's diagnostic entry point."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1908_03121_gb300 as F

pytestmark = pytest.mark.gpu


def _values():
    rng = np.random.default_rng(11)
    n = 1 << 20
    mag = 10.0 ** rng.uniform(-37.9, 38.5, n)
    v = mag * rng.choice([-1.0, 1.0], n)
    # exact float values, and values half an ulp away (ties of rounding to
    # nearest) and just either side of them
    f = rng.uniform(-1e6, 1e6, 4096).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(f).astype(np.float32)).astype(np.float64)
    ties = np.concatenate([f, f + ulp / 2, f - ulp / 2, f + ulp / 2 * (1 + 2 ** -20),
                           f + ulp / 2 * (1 - 2 ** -20)])
    fmax = float(np.finfo(np.float32).max)
    fmin = float(np.finfo(np.float32).tiny)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax,
                        fmax * (1 + 2 ** -25), fmax * (1 + 2 ** -23), fmin, -fmin, fmin * 1.5,
                        1.0, -1.0, 0.1, 1.0 / 3.0, 2.0 ** 100, 2.0 ** -100])
    # a NaN whose payload sits below the bits a float keeps
    special = np.concatenate([special, np.array([0x7FF0000000000001], dtype=np.uint64).view(np.float64)])
    return np.concatenate([v, ties, special])


def test_conversions_match_hardware():
    vals = torch.from_numpy(_values()).cuda()
    bad = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    F.fmm_check_conversions(vals, bad)
    torch.cuda.synchronize()
    assert int(bad.item()) == 0
