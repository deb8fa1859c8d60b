"""Explicit Runge-Kutta time stepping, FP64 (test infrastructure only).

The paper advances in time with a second-order scheme with adaptive steps
(Sec. 2.3) whose coefficients are not given; the workloads here use
classical RK4 (tiny vortex case) and the five-stage, fourth-order 2N-storage
scheme of Carpenter and Kennedy (1994) with a fixed step.  Adaptive steps
use, in place of the paper's scheme, the embedded 3(2) pair of Bogacki and
Shampine (1989) with its first-same-as-last stage and the elementary
error-per-step controller (Hairer, Norsett and Wanner, Solving ODEs I,
Sec. II.4): see ``AdaptiveBS32``.

2N-storage form, stage i = 1..5:
    dU <- A_i dU + dt R(u)
    u  <- u + B_i dU
with A_1 = 0 (so dU from the previous step is never read).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

LSRK45_A = [Fraction(0), Fraction(-567301805773, 1357537059087),
            Fraction(-2404267990393, 2016746695238),
            Fraction(-3550918686646, 2091501179385),
            Fraction(-1275806237668, 842570457699)]
LSRK45_B = [Fraction(1432997174477, 9575080441755),
            Fraction(5161836677717, 13612068292357),
            Fraction(1720146321549, 2090206949498),
            Fraction(3134564353537, 4481467310338),
            Fraction(2277821191437, 14882151754819)]

RK4_STAGES = 4
LSRK45_STAGES = 5


def rk4_step(rhs, u, dt):
    """Classical fourth-order Runge-Kutta."""
    k1 = rhs(u)
    k2 = rhs(u + 0.5 * dt * k1)
    k3 = rhs(u + 0.5 * dt * k2)
    k4 = rhs(u + dt * k3)
    return u + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def lsrk45_step(rhs, u, dt):
    """Carpenter-Kennedy 5-stage 4th-order 2N-storage step."""
    A = [float(a) for a in LSRK45_A]
    B = [float(b) for b in LSRK45_B]
    du = np.zeros_like(u)
    for i in range(5):
        du = A[i] * du + dt * rhs(u)
        u = u + B[i] * du
    return u


def step(rhs, u, dt, scheme):
    if scheme == "rk4":
        return rk4_step(rhs, u, dt)
    if scheme == "lsrk45":
        return lsrk45_step(rhs, u, dt)
    raise ValueError(scheme)


def lsrk45_butcher():
    """Equivalent Butcher tableau (a, b, c) of the 2N scheme, exact rationals.

    With k_j = R(u_{j-1}) the stage-j derivative, dU_i = sum_{j<=i}
    (prod_{m=j+1}^{i} A_m) dt k_j and u_i = u_0 + sum_{l<=i} B_l dU_l."""
    A, B = LSRK45_A, LSRK45_B
    s = 5
    a = [[Fraction(0)] * s for _ in range(s + 1)]
    for i in range(1, s + 1):          # row i: input of stage i+1 (row s: final)
        for j in range(1, i + 1):
            tot = Fraction(0)
            for l in range(j, i + 1):
                prod = Fraction(1)
                for m in range(j + 1, l + 1):
                    prod *= A[m - 1]
                tot += B[l - 1] * prod
            a[i][j - 1] = tot
    b = a[s]
    amat = a[:s]
    c = [sum(row) for row in amat]
    return amat, b, c


# ---------------------------------------------------------------------------
# Adaptive steps: Bogacki-Shampine 3(2) pair
# ---------------------------------------------------------------------------
# Butcher tableau, exact rationals.  The third-order weights b advance the
# solution (local extrapolation); the second-order weights bhat only serve
# the error estimate.  The last row of a equals b (first same as last): the
# fourth stage derivative R(u_{n+1}) is the first one of the next step.
BS32_A = [[Fraction(0)] * 4,
          [Fraction(1, 2), Fraction(0), Fraction(0), Fraction(0)],
          [Fraction(0), Fraction(3, 4), Fraction(0), Fraction(0)],
          [Fraction(2, 9), Fraction(1, 3), Fraction(4, 9), Fraction(0)]]
BS32_B = [Fraction(2, 9), Fraction(1, 3), Fraction(4, 9), Fraction(0)]
BS32_BHAT = [Fraction(7, 24), Fraction(1, 4), Fraction(1, 3), Fraction(1, 8)]
BS32_C = [Fraction(0), Fraction(1, 2), Fraction(3, 4), Fraction(1)]

# controller constants: safety factor, bounds of the step-size ratio, and the
# exponent -1/(qhat + 1) of the error of the embedded order qhat = 2
CTRL_SAFETY = 0.9
CTRL_FMIN = 0.2
CTRL_FMAX = 10.0
CTRL_EXPONENT = -1.0 / 3.0


def bs32_attempt(rhs, u, k1, h):
    """One Bogacki-Shampine step of size h from u with k1 = R(u).

    Returns (u_new, k4, e): the third-order solution, R(u_new) (the next
    step's k1) and the local error estimate e = h sum_i (bhat_i - b_i) k_i."""
    a = [[float(x) for x in row] for row in BS32_A]
    k = [k1]
    for i in range(1, 4):
        ui = u.copy()
        for j in range(i):
            if a[i][j] != 0.0:
                ui = ui + h * a[i][j] * k[j]
        if i == 3:
            u_new = ui
        k.append(rhs(ui))
    e = np.zeros_like(u)
    for i in range(4):
        e = e + h * float(BS32_BHAT[i] - BS32_B[i]) * k[i]
    return u_new, k[3], e


def error_norm(e, u, u_new, rtol, atol):
    """Root-mean-square over every value of e / (atol + rtol max(|u|, |u_new|));
    atol is a scalar or one value per variable (the last axis of u)."""
    scale = np.asarray(atol, dtype=np.float64) + rtol * np.maximum(np.abs(u), np.abs(u_new))
    r = e / scale
    return float(np.sqrt(np.mean(r * r)))


class AdaptiveBS32:
    """Adaptive integration of du/dt = rhs(u) with the Bogacki-Shampine pair.

    State: time t, proposed step h, the current solution u and k1 = R(u).
    One attempt (``attempt``):
      1. the step used is h_use = min(h, dt_max), shortened to end exactly
         at t_end (0 once t_end is reached: the attempt changes nothing);
      2. u_new, k4 and the error estimate from ``bs32_attempt``;
      3. err = ``error_norm``; accepted when err < 1;
      4. accepted: t += h_use, u = u_new, k1 = k4, and the next proposal is
         h_use * f with f = fmax (err = 0) or min(fmax, safety err^(-1/3)),
         capped at 1 when this step already had a rejected attempt;
         rejected: u and t stay, and the proposal is
         h_use * max(fmin, safety err^(-1/3)).
    """

    def __init__(self, rhs, u0, h0, t_end, rtol, atol, dt_max=np.inf, t0=0.0):
        self.rhs = rhs
        self.u = np.array(u0, dtype=np.float64)
        self.k1 = rhs(self.u)
        self.t = float(t0)
        self.h = float(h0)
        self.t_end = float(t_end)
        self.rtol = float(rtol)
        self.atol = atol
        self.dt_max = float(dt_max)
        self.rejected_in_step = False
        self.n_accepted = 0
        self.n_rejected = 0
        self.records = []

    def step_size(self):
        h = min(self.h, self.dt_max)
        if self.t + h > self.t_end:
            h = self.t_end - self.t
        return max(h, 0.0)

    def attempt(self):
        h = self.step_size()
        if h == 0.0:
            self.records.append(dict(t=self.t, h=0.0, err=0.0, accepted=False))
            return False
        u_new, k4, e = bs32_attempt(self.rhs, self.u, self.k1, h)
        err = error_norm(e, self.u, u_new, self.rtol, self.atol)
        accepted = err < 1.0
        self.records.append(dict(t=self.t, h=h, err=err, accepted=accepted))
        if accepted:
            f = CTRL_FMAX if err == 0.0 else min(CTRL_FMAX, CTRL_SAFETY * err ** CTRL_EXPONENT)
            if self.rejected_in_step:
                f = min(1.0, f)
            self.t = self.t + h if self.t + h < self.t_end else self.t_end
            self.u, self.k1 = u_new, k4
            self.h = h * f
            self.rejected_in_step = False
            self.n_accepted += 1
        else:
            self.h = h * max(CTRL_FMIN, CTRL_SAFETY * err ** CTRL_EXPONENT)
            self.rejected_in_step = True
            self.n_rejected += 1
        return accepted

    def run(self, n_attempts=None):
        """n_attempts attempts, or (None) attempts until t_end is reached."""
        if n_attempts is None:
            while self.t < self.t_end:
                self.attempt()
        else:
            for _ in range(n_attempts):
                self.attempt()
        return self.u
