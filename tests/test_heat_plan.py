"""Host-side plan of the heat-kernel Gibbs kernel (Sec. 4.1, Eq. heat-kernel),
read through jko_heat_plan without a GPU: the Chebyshev coefficients against
NumPy's Chebyshev interpolation of lambda^{-L}, the truncated series against
lambda^{-L} on the whole spectrum interval, the interval itself (the
Gershgorin bound of Id - (gamma/L) Delta), and the argument checks."""
import shutil

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C


@pytest.fixture(scope="module")
def jko():
    if shutil.which("nvcc") is None:
        pytest.skip("no CUDA toolkit to build libjko")
    from paper_1502_06216_gb300 import jko as mod
    return mod


CASES = [(100, 100, 5e-4, 10), (44, 44, 5e-4, 10), (40, 56, 5e-4, 10), (64, 64, 2e-3, 10),
         (256, 128, 5e-4, 4), (1, 64, 1e-3, 10), (5, 4, 1e-4, 10)]


@pytest.mark.parametrize("nx,ny,gamma,L", CASES)
@pytest.mark.parametrize("prec,eps", [("FP64", 2e-15), ("FP32", 2e-15)])
def test_plan_is_the_chebyshev_series_of_the_power(jko, nx, ny, gamma, L, prec, eps):
    plan = jko.jko_heat_plan(nx, ny, gamma, L, precision=jko.Precision[prec])
    lo, hi = plan["interval"]
    c = gamma / L
    assert lo == 1.0
    assert abs(hi - (1 + 4 * c * nx * nx + 4 * c * ny * ny)) <= 1e-12 * hi
    D, coef = plan["degree"], plan["coef"]
    assert 1 <= D <= 1500 and coef.size == D + 1
    f = lambda lam: lam ** (-float(L))
    ref = C.Chebyshev.interpolate(f, max(2 * D, 64), domain=[lo, hi]).coef
    assert np.abs(coef - ref[:D + 1]).max() <= 1e-13
    lam = np.linspace(lo, hi, 4001)
    series = C.Chebyshev(coef, domain=[lo, hi])(lam)
    err = np.abs(series - f(lam)).max()
    assert err <= 5 * eps, err
    # not far above the smallest degree that meets the target
    dmin = next(d for d in range(1, D + 1)
                if np.abs(C.Chebyshev(coef[:d + 1], domain=[lo, hi])(lam) - f(lam)).max() <= 5 * eps)
    assert D <= dmin + 12, (D, dmin)


def test_degrees_of_the_bench_and_test_grids(jko):
    # FP32 handles truncate where FP64 ones do (their recurrence runs in FP64)
    assert jko.jko_heat_plan(100, 100, 5e-4, 10, precision=jko.Precision.FP32)["degree"] == 54
    assert jko.jko_heat_plan(100, 100, 5e-4, 10, precision=jko.Precision.FP64)["degree"] == 54
    assert jko.jko_heat_plan(44, 44, 5e-4, 10, precision=jko.Precision.FP64)["degree"] == 26
    # a tiny interval (lmax ~ 1.0016): the series is short, its tail at the rounding floor
    assert jko.jko_heat_plan(5, 4, 1e-4, 10, precision=jko.Precision.FP64)["degree"] <= 8


def test_argument_checks(jko):
    for args in ((0, 10, 1e-3, 10), (10, 10, 0.0, 10), (10, 10, 1e-3, 0), (10, 10, 1e-3, 1001)):
        with pytest.raises(jko.JKOError):
            jko.jko_heat_plan(*args)
    with pytest.raises(jko.JKOError):
        jko.jko_heat_plan(10, 10, 1e-3, 10, precision=jko.Precision.BF16)
    with pytest.raises(jko.JKOError):                       # degree above 1500
        jko.jko_heat_plan(4096, 4096, 1.0, 1, precision=jko.Precision.FP64)
