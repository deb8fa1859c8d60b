"""Seeded initial conditions and free-stream data, as pointwise functions of
physical coordinates (the coordinates of the solution points are supplied by
the caller: the oracle and the CUDA library each compute their own).

State vectors are conserved variables [rho, rho*u_i, rho*E] (Sec. 2.1,
Eq. 2), non-dimensionalised with rho_inf = 1 and a reference speed of 1
unless stated otherwise.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def primitive_to_conserved(rho, vel, p, gamma=GAMMA):
    """Stack [rho, rho*v_i, p/(gamma-1) + 0.5*rho*|v|^2] along the last axis."""
    vel = np.asarray(vel)
    ke = 0.5 * rho * np.sum(vel * vel, axis=-1)
    mom = rho[..., None] * vel
    return np.concatenate([rho[..., None], mom, (p / (gamma - 1.0) + ke)[..., None]], -1)


def reference_conserved(dim, rho_inf=1.0, v_inf=None, p_inf=1.0, gamma=GAMMA):
    """Conserved free stream [rho, rho v, p/(gamma-1) + rho |v|^2 / 2]."""
    v = np.zeros(dim) if v_inf is None else np.asarray(v_inf, float)[:dim]
    return primitive_to_conserved(np.asarray(rho_inf, float), v, np.asarray(p_inf, float), gamma)


def fp32_perturbation_input(u, uref):
    """The state a mixed-precision (FP32) solver holds for the FP64 state u:
    it stores the FP32 rounding of u - u_ref, u_ref's components themselves
    rounded to FP32, so its arithmetic sees u_ref + fl32(u - u_ref)."""
    r = np.asarray(uref, float).astype(np.float32).astype(np.float64)
    return r + (u - r).astype(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# isentropic vortex (Shu's form; beta=5, M=0.5 in the tiny workload)
# ---------------------------------------------------------------------------

def vortex_speed(mach=0.5, gamma=GAMMA):
    """Advection speed of the vortex: free stream rho=p=1 so c=sqrt(gamma)."""
    return mach * np.sqrt(gamma)


def isentropic_vortex(x, t=0.0, beta=5.0, mach=0.5, gamma=GAMMA,
                      period=10.0, centre=(0.0, 0.0)):
    """Exact advected vortex at time t on a periodic box of side ``period``.

    The initial field is sampled on the fundamental cell [-period/2,
    period/2)^2 and the solution at time t is that field translated by the
    free stream (the periodic-image mismatch is below e^-12)."""
    x = np.asarray(x, float)
    u_inf = vortex_speed(mach, gamma)
    half = 0.5 * period
    xr = x[..., 0] - centre[0] - u_inf * t
    yr = x[..., 1] - centre[1]
    xr = (xr + half) % period - half
    yr = (yr + half) % period - half
    r2 = xr * xr + yr * yr
    f = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2.0 * np.pi) * yr * f
    dv = beta / (2.0 * np.pi) * xr * f
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2) * f * f
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    vel = np.stack([u_inf + du, dv], -1)
    return primitive_to_conserved(rho, vel, p, gamma)


# ---------------------------------------------------------------------------
# Taylor-Green vortex (Re=1600, M=0.1)
# ---------------------------------------------------------------------------

def taylor_green(x, mach=0.1, gamma=GAMMA):
    """TGV initial field, isothermal start with rho0 = 1, U0 = 1."""
    x = np.asarray(x, float)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    p0 = 1.0 / (gamma * mach * mach)
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = p / p0
    return primitive_to_conserved(rho, np.stack([u, v, w], -1), p, gamma)


# ---------------------------------------------------------------------------
# free stream and seeded perturbations
# ---------------------------------------------------------------------------

def free_stream(shape, dim, mach, gamma=GAMMA, direction=None):
    """Uniform flow rho=1, |v|=1, p=1/(gamma M^2) broadcast to ``shape``."""
    d = np.zeros(dim)
    d[0] = 1.0
    if direction is not None:
        d = np.asarray(direction, float)
        d = d / np.linalg.norm(d)
    rho = np.ones(shape)
    vel = np.broadcast_to(d, tuple(shape) + (dim,))
    p = np.full(shape, 1.0 / (gamma * mach * mach))
    return primitive_to_conserved(rho, vel, p, gamma)


def smooth_perturbed(x, dim, mach, amp=0.05, seed=2312, n_modes=4, gamma=GAMMA):
    """Free stream plus a seeded sum of smooth Fourier modes in rho, v, p.

    Produces states with O(amp) relative variation that keep density and
    pressure positive; used as parity inputs on non-periodic meshes."""
    rng = np.random.default_rng(seed)
    x = np.asarray(x, float)
    shp = x.shape[:-1]
    p_inf = 1.0 / (gamma * mach * mach)
    prim = [np.ones(shp)] + [np.zeros(shp) for _ in range(dim)] + [np.full(shp, p_inf)]
    prim[1] = prim[1] + 1.0
    scale = [1.0] + [1.0] * dim + [p_inf]
    for comp in range(dim + 2):
        acc = np.zeros(shp)
        for _ in range(n_modes):
            k = rng.uniform(0.2, 1.5, size=dim) * rng.choice([-1, 1], size=dim)
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.uniform(0.3, 1.0)
            acc += a * np.sin(x @ k + ph)
        prim[comp] = prim[comp] + amp * scale[comp] * acc / n_modes
    rho, p = prim[0], prim[-1]
    vel = np.stack(prim[1:1 + dim], -1)
    return primitive_to_conserved(rho, vel, p, gamma)


def random_state(n_elem, n_sp, dim, mach, amp=0.05, seed=2312, gamma=GAMMA):
    """Free stream with independent seeded nodal noise (rough, non-smooth),
    layout (n_elem, n_sp, dim+2)."""
    rng = np.random.default_rng(seed)
    shp = (n_elem, n_sp)
    rho = 1.0 + amp * rng.uniform(-1, 1, shp)
    vel = np.zeros(shp + (dim,))
    vel[..., 0] = 1.0
    vel = vel + amp * rng.uniform(-1, 1, shp + (dim,))
    p = (1.0 / (gamma * mach * mach)) * (1.0 + amp * rng.uniform(-1, 1, shp))
    return primitive_to_conserved(rho, vel, p, gamma)


def wall_damped(x, wall_pts, delta, base):
    """Scale the velocity of the conserved state ``base`` by
    1 - exp(-d/delta), d the distance of each point to the nearest of the
    ``wall_pts`` (a dense sampling of the wall), keeping density and
    pressure: a start that satisfies the no-slip wall instead of an
    impulsive one."""
    from scipy.spatial import cKDTree
    x = np.asarray(x, float)
    d, _ = cKDTree(np.asarray(wall_pts, float)).query(x.reshape(-1, x.shape[-1]))
    f = (1.0 - np.exp(-d / delta)).reshape(x.shape[:-1])
    dim = x.shape[-1]
    rho = base[..., 0]
    vel = base[..., 1:1 + dim] / rho[..., None]
    p = (GAMMA - 1.0) * (base[..., -1] - 0.5 * rho * np.sum(vel * vel, -1))
    return primitive_to_conserved(rho, vel * f[..., None], p)
