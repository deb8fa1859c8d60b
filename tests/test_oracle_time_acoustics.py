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


# ---------------------------------------------------------------------------
# Adaptive steps (Bogacki-Shampine 3(2) pair, elementary controller)
# ---------------------------------------------------------------------------

def test_bs32_tableau_orders_exact():
    """b meets every condition of order 3, bhat those of order 2 but not the
    order-3 ones (so the difference estimates the error); the rows of a sum
    to c; the last row of a is b with c = 1 (first same as last)."""
    a, b, bh, c = timestep.BS32_A, timestep.BS32_B, timestep.BS32_BHAT, timestep.BS32_C
    s = 4
    for i in range(s):
        assert sum(a[i]) == c[i]
        assert all(a[i][j] == 0 for j in range(i, s))     # explicit
    assert a[3] == b and c[3] == 1
    ac = [sum(a[i][j] * c[j] for j in range(s)) for i in range(s)]
    assert sum(b) == 1 and sum(b[i] * c[i] for i in range(s)) == Fraction(1, 2)
    assert sum(b[i] * c[i] ** 2 for i in range(s)) == Fraction(1, 3)
    assert sum(b[i] * ac[i] for i in range(s)) == Fraction(1, 6)
    assert sum(bh) == 1 and sum(bh[i] * c[i] for i in range(s)) == Fraction(1, 2)
    third = (sum(bh[i] * c[i] ** 2 for i in range(s)) - Fraction(1, 3),
             sum(bh[i] * ac[i] for i in range(s)) - Fraction(1, 6))
    assert third != (0, 0)


def test_bs32_error_estimate_is_third_order_on_the_linear_equation():
    """For y' = lambda y the estimate is h lambda (R(z) - Rhat(z)) y with
    R - Rhat = O(z^3): halving h divides it by 8 in the limit, and the
    third-order solution matches exp(z) to O(z^4)."""
    lam = -1.3
    ests, errs = [], []
    for h in (0.08, 0.04, 0.02, 0.01):
        u = np.array([1.0])
        un, _, e = timestep.bs32_attempt(lambda y: lam * y, u, lam * u, h)
        ests.append(abs(e[0]))
        errs.append(abs(un[0] - math.exp(lam * h)))
    r_est = [ests[i] / ests[i + 1] for i in range(3)]
    r_err = [errs[i] / errs[i + 1] for i in range(3)]
    assert abs(r_est[-1] - 8.0) < 0.2
    assert abs(r_err[-1] - 16.0) < 0.5


def _lotka(y):
    return np.array([1.5 * y[0] - y[0] * y[1], -3.0 * y[1] + y[0] * y[1]])


def test_adaptive_bs32_matches_scipy_rk23_on_an_ode():
    """scipy's RK23 integrates with the same pair and the same elementary
    controller: the accepted times and solution agree to rounding, through
    a deliberately oversized first step (rejections) and the final step cut
    to end on t_end."""
    integrate = pytest.importorskip("scipy.integrate")
    y0 = np.array([2.0, 1.0])
    rtol, atol, h0, t_end = 1e-6, 1e-9, 0.5, 3.0
    ad = timestep.AdaptiveBS32(_lotka, y0, h0, t_end, rtol, atol)
    ad.run()
    ref = integrate.solve_ivp(lambda t, y: _lotka(y), (0.0, t_end), y0, method="RK23",
                              rtol=rtol, atol=atol, first_step=h0)
    assert ref.status == 0
    acc_t = [0.0] + [r["t"] + r["h"] for r in ad.records if r["accepted"]]
    acc_t[-1] = ad.t
    assert ad.n_rejected >= 1
    assert len(acc_t) == ref.t.size
    assert np.max(np.abs(np.array(acc_t) - ref.t)) < 1e-12 * t_end
    assert np.max(np.abs(ad.u - ref.y[:, -1])) < 1e-10
    assert ad.t == t_end


def test_adaptive_bs32_matches_scipy_rk23_on_the_fr_semidiscretisation():
    """The same agreement with the FR residual of a small isentropic vortex
    (Euler, p = 2) as right-hand side, with one absolute tolerance per
    conserved variable and a step cap."""
    integrate = pytest.importorskip("scipy.integrate")
    from tests import fr_cases as FC
    case = FC.vortex_case(n=4, p=2)
    disc = FC.oracle_disc(case)
    u0 = FC.initial_state(case, disc.sol_coords())
    shape = u0.shape
    atol = np.array([1e-6, 1e-6, 1e-6, 1e-5])
    rtol, h0, t_end, dt_max = 1e-5, 0.2, 0.3, 0.05
    ad = timestep.AdaptiveBS32(disc.residual, u0, h0, t_end, rtol, atol, dt_max=dt_max)
    ad.run()

    def f(t, y):
        return disc.residual(y.reshape(shape)).ravel()
    ref = integrate.solve_ivp(f, (0.0, t_end), u0.ravel(), method="RK23", rtol=rtol,
                              atol=np.broadcast_to(atol, shape).ravel(), first_step=h0,
                              max_step=dt_max)
    assert ref.status == 0
    n_acc = sum(r["accepted"] for r in ad.records)
    assert ad.n_rejected >= 1 and n_acc + 1 == ref.t.size
    acc_t = np.cumsum([r["h"] for r in ad.records if r["accepted"]])
    assert np.max(np.abs(acc_t - ref.t[1:])) < 1e-12
    assert np.max(np.abs(ad.u.ravel() - ref.y[:, -1])) < 1e-11


def test_adaptive_run_at_the_stability_limit_is_sensitive_to_rounding():
    """Why the GPU compares the Taylor-Green 4^3 adaptive run over its first
    16 attempts only: the oracle run twice, once with its residual perturbed
    by 1e-14 relative (rounding-sized), agrees to 1e-7 in the error norm
    through attempt 16, but once the steps ride the stability limit the
    difference grows by orders of magnitude (above 1e-4 by attempt 30).  The
    periodic 2-D case, whose steps stay accuracy-limited, keeps it below
    1e-8 to its end."""
    from tests import fr_cases as FC

    def drift(case, h0, t_end, rtol, atol, n):
        disc = FC.oracle_disc(case)
        u0 = FC.initial_state(case, disc.sol_coords())
        rng = np.random.default_rng(1)

        def noisy(u):
            r = disc.residual(u)
            return r * (1.0 + 1e-14 * rng.standard_normal(r.shape))
        a = timestep.AdaptiveBS32(disc.residual, u0, h0, t_end, rtol, np.asarray(atol))
        b = timestep.AdaptiveBS32(noisy, u0, h0, t_end, rtol, np.asarray(atol))
        out = []
        while len(out) < n and a.t < t_end and b.t < t_end:
            a.attempt()
            b.attempt()
            ea, eb = a.records[-1]["err"], b.records[-1]["err"]
            out.append(abs(ea - eb) / ea)
        return np.array(out)

    tgv = drift(FC.tgv_case(n=4, p=3), 0.05, 0.3, 1e-4, [1e-5] * 5, 30)
    assert tgv.size == 30 and tgv[:16].max() < 1e-7 and tgv[24:].max() > 1e-4
    pns = drift(FC.periodic_ns_case(n=4, p=3), 0.04, 0.12, 1e-6, [1e-7] * 4, 100)
    assert pns.max() < 1e-8
