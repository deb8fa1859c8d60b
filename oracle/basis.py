"""One-dimensional building blocks of the FR reference element, in FP64.

Test infrastructure only: nothing in the product path imports this module.

* Gauss-Legendre solution points and weights (the point set the tiny
  isentropic-vortex workload names: n = p+1 Gauss-Legendre points).
* Lagrange interpolation and differentiation on those points.
* The DG-recovery ("g_DG") correction functions of Huynh's FR (the method of
  Sec. 2.3): g_L is the right Radau polynomial of degree p+1 and g_R its
  mirror image, g_L(-1) = 1, g_L(1) = 0, g_R(-1) = 0, g_R(1) = 1.
"""
from __future__ import annotations

import numpy as np


def legendre(k: int, x):
    """P_k(x) and P_k'(x) via Bonnet's recurrence
    (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}, and
    P'_{n+1} = P'_{n-1} + (2n+1) P_n."""
    x = np.asarray(x, dtype=np.float64)
    p_prev, p = np.ones_like(x), x.copy()
    d_prev, d = np.zeros_like(x), np.ones_like(x)
    if k == 0:
        return p_prev, d_prev
    for n in range(1, k):
        p_next = ((2 * n + 1) * x * p - n * p_prev) / (n + 1)
        d_next = d_prev + (2 * n + 1) * p
        p_prev, p = p, p_next
        d_prev, d = d, d_next
    return p, d


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1]: ascending nodes (roots of P_n,
    found by Newton's method) and weights w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2)."""
    if n < 1:
        raise ValueError("n >= 1")
    i = np.arange(n)
    x = -np.cos(np.pi * (i + 0.75) / (n + 0.5))
    for _ in range(100):
        p, dp = legendre(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dp = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def lagrange(nodes, x):
    """L[i, j] = l_j(x_i): the j-th Lagrange basis polynomial on ``nodes``
    evaluated at the points ``x``."""
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    n = nodes.size
    L = np.ones((x.size, n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_deriv(nodes, x):
    """dL[i, j] = l_j'(x_i), by differentiating the product form term by term."""
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    n = nodes.size
    dL = np.zeros((x.size, n))
    for j in range(n):
        denom = 1.0
        for m in range(n):
            if m != j:
                denom *= nodes[j] - nodes[m]
        for r in range(n):
            if r == j:
                continue
            term = np.ones(x.size)
            for m in range(n):
                if m != j and m != r:
                    term *= x - nodes[m]
            dL[:, j] += term
        dL[:, j] /= denom
    return dL


def correction_dg(p: int, x):
    """DG-recovery correction functions and their derivatives at x:
    g_L = (-1)^{p+1}/2 (P_{p+1} - P_p), g_R = 1/2 (P_{p+1} + P_p).
    Returns (gL, gR, dgL, dgR)."""
    P1, dP1 = legendre(p + 1, x)
    P0, dP0 = legendre(p, x)
    s = (-1.0) ** (p + 1) / 2.0
    return s * (P1 - P0), 0.5 * (P1 + P0), s * (dP1 - dP0), 0.5 * (dP1 + dP0)
