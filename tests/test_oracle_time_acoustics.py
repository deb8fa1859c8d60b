"""Pins of the oracle's time integrators and OASPL reduction.

* LSRK45: the equivalent Butcher tableau satisfies all eight fourth-order
  conditions exactly in rational arithmetic (a transcription error in any
  coefficient breaks at least one); RK4 reproduces the degree-4 Taylor
  polynomial of exp(z).
* OASPL (Sec. 3.1.2, Eqs. 9-12): closed forms for constant and sinusoidal
  signals, brute-force rational arithmetic for the running-mean reading.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import timestep, acoustics


def test_lsrk45_order_conditions_exact():
    a, b, c = timestep.lsrk45_butcher()
    s = len(b)
    one = Fraction(1)
    # consistency of c with the rows of a
    assert c[0] == 0
    ac = [sum(a[i][j] * c[j] for j in range(s)) for i in range(s)]
    ac2 = [sum(a[i][j] * c[j] ** 2 for j in range(s)) for i in range(s)]
    aac = [sum(a[i][j] * ac[j] for j in range(s)) for i in range(s)]
    conds = {
        "b": (sum(b), one),
        "bc": (sum(b[i] * c[i] for i in range(s)), Fraction(1, 2)),
        "bc2": (sum(b[i] * c[i] ** 2 for i in range(s)), Fraction(1, 3)),
        "bac": (sum(b[i] * ac[i] for i in range(s)), Fraction(1, 6)),
        "bc3": (sum(b[i] * c[i] ** 3 for i in range(s)), Fraction(1, 4)),
        "bcac": (sum(b[i] * c[i] * ac[i] for i in range(s)), Fraction(1, 8)),
        "bac2": (sum(b[i] * ac2[i] for i in range(s)), Fraction(1, 12)),
        "baac": (sum(b[i] * aac[i] for i in range(s)), Fraction(1, 24)),
    }
    for name, (got, want) in conds.items():
        # the published coefficients are 13-digit rationals: the conditions
        # hold to about 1e-12, far below any transcription error
        assert abs(float(got - want)) < 1e-11, name


def _stability_poly(step, order=6):
    """Coefficients of the amplification factor R(z) for y' = z y, by
    evaluating one step on polynomials in z."""
    P = np.polynomial.Polynomial

    def rhs(u):
        return u * P([0, 1])
    out = step(rhs, P([1.0]), 1.0)
    return np.pad(out.coef, (0, max(0, order - out.coef.size)))


@pytest.mark.parametrize("step", [timestep.rk4_step, timestep.lsrk45_step])
def test_stability_polynomial_matches_exp_to_fourth_order(step):
    coef = _stability_poly(step)
    for k in range(5):
        assert abs(coef[k] - 1.0 / math.factorial(k)) < 1e-12


def test_oaspl_constant_signal_is_minus_infinity_and_zero_rms():
    sig = np.full(100, 3.25)
    assert acoustics.p_rms(sig, mode=1) == 0.0
    assert acoustics.p_rms(sig, mode=0) == 0.0
    assert acoustics.oaspl(sig, mode=1) == -np.inf


def test_oaspl_sinusoid_window_mode_closed_form():
    n_per, periods = 64, 10
    t = np.arange(n_per * periods) / n_per
    A, B = 7.0, 0.03
    sig = A + B * np.sin(2 * np.pi * t)
    assert abs(acoustics.p_rms(sig, mode=1) - B / math.sqrt(2)) < 1e-14
    db = acoustics.oaspl(sig, mode=1, p_ref=2e-5, p_scale=10.0)
    assert abs(db - 20 * math.log10(10.0 * B / math.sqrt(2) / 2e-5)) < 1e-10
    # 0.1 dB corresponds to a 1.16 % change in p_RMS
    assert abs(20 * math.log10(1.0116) - 0.1) < 1e-3


def test_oaspl_running_mode_brute_force_rational():
    rng = np.random.default_rng(7)
    vals = rng.integers(-50, 50, size=60)
    sig = 100.0 + vals / 8.0
    F = [Fraction(int(v), 8) + 100 for v in vals]
    n = len(F)
    tot = Fraction(0)
    run = Fraction(0)
    for i, pi in enumerate(F, start=1):
        run += pi
        pbar = run / i
        tot += (pi - pbar) ** 2
    exact = math.sqrt(float(tot / n))
    assert abs(acoustics.p_rms(sig, mode=0) - exact) < 1e-13
    # the running mean differs from the window mean
    assert abs(acoustics.p_rms(sig, mode=1) - exact) > 1e-6


def test_oaspl_multi_probe_averages_rms_then_converts():
    a = np.sin(np.linspace(0, 20 * np.pi, 2000, endpoint=False))
    b = 3.0 * a
    db = acoustics.oaspl([a, b], mode=1, p_ref=1.0)
    want = 20 * math.log10(2.0 / math.sqrt(2))
    assert abs(db - want) < 1e-10
