"""Explicit Runge-Kutta time stepping, FP64 (test infrastructure only).

The paper advances in time with a second-order scheme with adaptive steps
(Sec. 2.3) whose coefficients are not given; the workloads here use
classical RK4 (tiny vortex case) and the five-stage, fourth-order 2N-storage
scheme of Carpenter and Kennedy (1994) with a fixed step.

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
