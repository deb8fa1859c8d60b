"""Observer probe and OASPL, FP64 (test infrastructure only).

Sec. 3.1.2 defines the objective:
  OASPL = 20 log10(p_RMS / p_ref)                                (Eq. 9)
  p_RMS = sqrt(sum_{i=1..n} p'_i^2 / n)                          (Eq. 10)
  p' = p - p_bar                                                 (Eq. 11)
  p_bar_k = sum_{i<=k} p_i / k, k = 1..n                         (Eq. 12)
where p_bar, p' and p_RMS are vectors indexed by the number of samples and the
OASPL uses the last entry of p_RMS.  Read literally (mode 0, "running"),
p'_i = p_i - p_bar_i uses the cumulative mean up to sample i; mode 1
("window") subtracts the mean of the whole window, the ordinary RMS.  With
several observers along the span, p_RMS of each observer is computed and the
arithmetic mean of those values enters Eq. 9 once.  The solver is
non-dimensional, so p_RMS is multiplied by ``p_scale`` (Pa per solver unit)
before dividing by ``p_ref`` (the paper gives no value; 2e-5 Pa is used).

Probe sampling: the conserved variables are interpolated to the observer with
the element's tensor Lagrange basis and the pressure is computed from the
interpolated state.
"""
from __future__ import annotations

import numpy as np

from .geometry import jacobian, map_points


def p_rms(samples, mode=0):
    p = np.asarray(samples, dtype=np.float64)
    n = p.size
    if n == 0:
        return 0.0
    if mode == 0:
        pbar = np.cumsum(p) / np.arange(1, n + 1)
        pp = p - pbar
    elif mode == 1:
        pp = p - p.sum() / n
    else:
        raise ValueError("mode")
    return float(np.sqrt(np.sum(pp * pp) / n))


def oaspl(sample_sets, mode=0, p_ref=2e-5, p_scale=1.0):
    """OASPL in dB from one or several observers' pressure histories."""
    if np.ndim(sample_sets[0]) == 0:
        sample_sets = [sample_sets]
    prms = np.mean([p_rms(s, mode) for s in sample_sets])
    if prms == 0.0:
        return -np.inf
    return 20.0 * np.log10(p_scale * prms / p_ref)


def locate(mesh, ref, x_obs, tol=1e-13, max_iter=50):
    """(element, reference coordinates) of a physical point, by Newton's
    method on each element map whose node bounding box contains the point."""
    x_obs = np.asarray(x_obs, float)
    nodes = mesh.node_coords()
    lo = nodes.min(axis=1)
    hi = nodes.max(axis=1)
    pad = 1e-9 * (hi - lo).max(axis=1, keepdims=True)
    cand = np.nonzero(np.all((x_obs >= lo - pad) & (x_obs <= hi + pad), axis=1))[0]
    for e in cand:
        xi = np.zeros(mesh.dim)
        for _ in range(max_iter):
            x = map_points(mesh, [e], xi[None, :])[0, 0]
            A = jacobian(mesh, [e], xi[None, :])[0, 0]
            dxi = np.linalg.solve(A, x_obs - x)
            xi = xi + dxi
            if np.max(np.abs(xi)) > 3.0:
                break
            if np.max(np.abs(dxi)) < tol:
                break
        if np.all(np.abs(xi) <= 1.0 + 1e-10):
            return int(e), np.clip(xi, -1.0, 1.0)
    raise ValueError("observer outside the mesh")


class Probe:
    def __init__(self, disc, x_obs):
        self.elem, self.xi = locate(disc.mesh, disc.ref, x_obs)
        self.w = disc.ref.interp_matrix(self.xi[None, :])[0]          # (nsp,)
        self.phys = disc.phys

    def state(self, U):
        return self.w @ U[self.elem]

    def pressure(self, U):
        return float(self.phys.pressure(self.state(U)[None, :])[0])
