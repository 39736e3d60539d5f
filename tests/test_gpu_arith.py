"""Error bounds of the device arithmetic building blocks (needs a GB300).

The Gram solves of Algorithm 2 and the factorisations of the QR steps of
Algorithm 1 rest on double-word FP32 arithmetic (an unevaluated sum hi + lo of
two floats) and on an FP64 reciprocal square root refined from the FP32
estimate.  Each block is evaluated on the GPU through ``rcp_test_arith`` and
compared with exact rational arithmetic (``fractions``) or 60-digit decimals
on the host:

* sum (Joldes, Muller & Popescu 2017, AccurateDWPlusDW): <= 3u^2 + 13u^3,
* product (their DWTimesDW2, the form with the lo*lo term): <= 5u^2,
* reciprocal (Newton from the hardware estimate) and square root (one
  Karp-Markstein correction): <= 8u^2, "a few u^2",
* FP64 reciprocal square root: <= 2 ulp of FP64 (2^-51 relative),

with u = 2^-24.  Inputs span many binades, both signs for the sum (with
near-cancellation), and the FP64 routine's range-guard branch.
"""

import ctypes
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
N = 3000


def _dw_input(x):
    """The device's rounding of a double to its nearest double word."""
    hi = np.float32(x)
    lo = np.float32(np.float64(x) - np.float64(hi))
    return Fraction(float(hi)) + Fraction(float(lo))


def _run(op, x, y=None):
    from paper_1703_09074_gb300 import _lib
    lib = _lib.load()
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda() if y is not None else None
    hi = torch.empty_like(xd)
    lo = torch.empty_like(xd)
    st = lib.rcp_test_arith(op, ctypes.c_void_p(xd.data_ptr()),
                            ctypes.c_void_p(yd.data_ptr()) if yd is not None else None,
                            len(x), ctypes.c_void_p(hi.data_ptr()), ctypes.c_void_p(lo.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return hi.cpu().numpy(), lo.cpu().numpy()


def _magnitudes(rng, n, lo_exp=-30, hi_exp=30):
    return np.exp2(rng.uniform(lo_exp, hi_exp, n)) * rng.uniform(1.0, 2.0, n)


def _rel(got, exact):
    return abs(got - exact) / abs(exact)


def test_double_word_sum_and_product():
    from paper_1703_09074_gb300._lib import RCP_ARITH_DW_ADD, RCP_ARITH_DW_MUL
    rng = np.random.default_rng(1)
    x = _magnitudes(rng, N) * rng.choice([-1.0, 1.0], N)
    y = _magnitudes(rng, N) * rng.choice([-1.0, 1.0], N)
    # a third of the pairs nearly cancel: y = -x (1 + small)
    k = N // 3
    y[:k] = -x[:k] * (1.0 + rng.uniform(-1e-6, 1e-6, k))
    hi, lo = _run(RCP_ARITH_DW_ADD, x, y)
    worst = 0.0
    for i in range(N):
        exact = _dw_input(x[i]) + _dw_input(y[i])
        got = Fraction(float(hi[i])) + Fraction(float(lo[i]))
        if exact == 0:
            assert got == 0
            continue
        worst = max(worst, float(_rel(got, exact)))
        assert abs(lo[i]) <= abs(hi[i]) * U * 1.0000001 or hi[i] == 0  # normalised
    assert worst <= 3 * U ** 2 + 13 * U ** 3, worst
    hi, lo = _run(RCP_ARITH_DW_MUL, x, y)
    worst = 0.0
    for i in range(N):
        exact = _dw_input(x[i]) * _dw_input(y[i])
        got = Fraction(float(hi[i])) + Fraction(float(lo[i]))
        worst = max(worst, float(_rel(got, exact)))
    assert worst <= 5 * U ** 2, worst


def test_double_word_reciprocal_and_square_root():
    from paper_1703_09074_gb300._lib import RCP_ARITH_DW_RCP, RCP_ARITH_DW_SQRT
    rng = np.random.default_rng(2)
    x = _magnitudes(rng, N, -60, 60)
    hi, lo = _run(RCP_ARITH_DW_RCP, x)
    worst = 0.0
    for i in range(N):
        exact = 1 / _dw_input(x[i])
        got = Fraction(float(hi[i])) + Fraction(float(lo[i]))
        worst = max(worst, float(_rel(got, exact)))
    assert worst <= 8 * U ** 2, worst
    getcontext().prec = 60
    hi, lo = _run(RCP_ARITH_DW_SQRT, x)
    worst = Decimal(0)
    for i in range(N):
        a = _dw_input(x[i])
        exact = (Decimal(a.numerator) / Decimal(a.denominator)).sqrt()
        got = Decimal(float(hi[i])) + Decimal(float(lo[i]))
        worst = max(worst, abs(got - exact) / exact)
    assert worst <= Decimal(8 * U ** 2), worst


def test_fp64_reciprocal_square_root():
    from paper_1703_09074_gb300._lib import RCP_ARITH_RSQRT64
    rng = np.random.default_rng(3)
    # inside the refined range and beyond the exponent guard (|log2| > 99)
    x = np.concatenate([_magnitudes(rng, N, -95, 95), _magnitudes(rng, 200, 100, 900),
                        _magnitudes(rng, 200, -900, -100)])
    hi, lo = _run(RCP_ARITH_RSQRT64, x)
    assert np.all(lo == 0.0)
    getcontext().prec = 60
    worst = Decimal(0)
    for i in range(len(x)):
        exact = 1 / Decimal(float(x[i])).sqrt()
        worst = max(worst, abs(Decimal(float(hi[i])) - exact) / exact)
    assert worst <= Decimal(2.0 ** -51), worst


@pytest.mark.gpu
def test_fma_rate_measurement():
    """The FMA-rate kernel behind the FP64 path's roofline peak: positive rates, and
    FP32 well above FP64 on this part (FP64 issues at a small fraction of FP32)."""
    from paper_1703_09074_gb300 import measure_fma_rate
    f64 = measure_fma_rate(fp64=True)
    f32 = measure_fma_rate(fp64=False)
    assert f64 > 0.1 and f32 > 10.0 * f64
