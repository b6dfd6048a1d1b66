"""The integer-pipe FP64 FMA equals the hardware fma bit for bit."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


def cases(rng, n):
    a = rng.normal(size=n) * 2.0 ** rng.integers(-60, 60, n)
    b = rng.normal(size=n) * 2.0 ** rng.integers(-60, 60, n)
    c = rng.normal(size=n) * 2.0 ** rng.integers(-130, 130, n)
    k = n // 8
    # near-cancellation: c close to -a*b (exactly representable product parts)
    c[:k] = -(a[:k] * b[:k]) * (1 + rng.integers(-4, 5, k) * 2.0 ** -52)
    # exact ties: operands with few significant bits
    a[k:2 * k] = rng.integers(1, 2 ** 27, k) * 2.0 ** -26
    b[k:2 * k] = rng.integers(1, 2 ** 27, k) * 2.0 ** -26
    c[k:2 * k] = rng.integers(-2 ** 20, 2 ** 20, k) * 2.0 ** -70
    # zeros and signed zeros
    a[2 * k:2 * k + 64] = 0.0
    b[2 * k + 64:2 * k + 128] = -0.0
    c[2 * k + 128:2 * k + 256] = rng.choice([0.0, -0.0], 128)
    # the solver's regime: values and vectors of order one
    a[3 * k:4 * k] = rng.uniform(-1, 1, k)
    b[3 * k:4 * k] = rng.uniform(-2, 2, k)
    c[3 * k:4 * k] = rng.uniform(-3, 3, k)
    # subnormal, huge and special values (hardware fallback)
    a[4 * k:4 * k + 8] = [np.inf, -np.inf, np.nan, 5e-324, 1e308, 1e-310, 2.0, 3.0]
    b[4 * k:4 * k + 8] = [1.0, 0.0, 2.0, 3.0, 1e10, 1e-10, 1e308, 5e-324]
    return a, b, c


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fma64_int_is_bit_exact(bbs, seed):
    rng = np.random.default_rng(seed)
    a, b, c = cases(rng, 1 << 20)
    ta, tb, tc = (torch.as_tensor(v, device="cuda") for v in (a, b, c))
    got = bbs.bbs_fma64_int(ta, tb, tc)
    ref = torch.addcmul(tc, ta, tb)  # one fused rounding on the GPU's FP64 unit
    g = got.cpu().numpy().view(np.int64)
    r = ref.cpu().numpy().view(np.int64)
    nan = np.isnan(ref.cpu().numpy())
    bad = np.nonzero((g != r) & ~nan)[0]
    assert bad.size == 0, [(a[i], b[i], c[i], g[i], r[i]) for i in bad[:5]]
    assert np.isnan(got.cpu().numpy()[nan]).all()
