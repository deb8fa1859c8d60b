"""Shared set-up for the parity tests: one synthetic case built twice, once
through the CUDA library (C ABI via the thin binding) and once through the
FP64 oracle, from the same seeded mesh and state.  The two sides share only
the inputs (``synth``)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from synth import meshes as M, states as S

GAMMA = 1.4
PR = 0.71


@dataclass
class Case:
    name: str
    meshes: list
    p: int
    viscous: bool
    mu: float
    mach: float
    rk: str = "lsrk45"
    dt: float = 1e-3
    v_inf: tuple = (1.0, 0.0)
    inflow_delta: float = 0.0
    inflow_ywall: float = 0.0
    flux: str = "rusanov"
    viscous_scheme: str = "br2"
    p_ref: float = 0.0             # free-stream pressure if not 1/(gamma M^2)

    @property
    def dim(self):
        return self.meshes[0].dim

    @property
    def p_inf(self):
        return self.p_ref if self.p_ref > 0 else 1.0 / (GAMMA * self.mach ** 2)


def oracle_disc(case: Case, inst: int = 0):
    from oracle.fr import FRDiscretisation
    from oracle.physics import NavierStokes
    ph = NavierStokes(case.dim, gamma=GAMMA, mu=case.mu, prandtl=PR, viscous=case.viscous,
                      rho_inf=1.0, v_inf=case.v_inf[:case.dim], p_inf=case.p_inf,
                      inflow_delta=case.inflow_delta, inflow_ywall=case.inflow_ywall,
                      flux=case.flux)
    return FRDiscretisation(case.meshes[inst], case.p, ph, viscous_scheme=case.viscous_scheme)


def lib_config(case: Case, precision: str):
    from paper_2312_14167_gb300 import fr
    return fr.make_config(case.dim, gamma=GAMMA, prandtl=PR, mu=case.mu, rho_inf=1.0,
                          v_inf=case.v_inf, p_inf=case.p_inf, inflow_delta=case.inflow_delta,
                          inflow_ywall=case.inflow_ywall, dt=case.dt, viscous=case.viscous,
                          rk=fr.FR_RK4 if case.rk == "rk4" else fr.FR_LSRK45,
                          precision=fr.FR_FP64 if precision == "fp64" else fr.FR_FP32,
                          flux=fr.FR_FLUX_ROE if case.flux == "roe" else fr.FR_FLUX_RUSANOV,
                          viscous_scheme=fr.FR_VISC_LDG if case.viscous_scheme == "ldg" else fr.FR_VISC_BR2)


def lib_solver(case: Case, precision: str):
    from paper_2312_14167_gb300 import fr
    ms = [fr.Mesh(m, case.p) for m in case.meshes]
    return fr.Solver(ms, lib_config(case, precision))


def initial_state(case: Case, x, inst: int = 0):
    """Seeded smooth state at physical points x (shape (..., dim))."""
    info = case.meshes[inst].info
    if case.name.startswith("vortex"):
        return S.isentropic_vortex(x)
    if case.name.startswith("tgv"):
        return S.taylor_green(x, mach=case.mach)
    u = S.smooth_perturbed(x, case.dim, case.mach, amp=0.05, seed=100 + inst)
    if "wall_points" in info:
        u = S.wall_damped(x, info["wall_points"], 0.05, u)
    return u


def cfl_dt(meshes, mach, p, cfl=0.4):
    """Fixed step from a CFL estimate on the corner-edge lengths."""
    c = np.sqrt(GAMMA / (GAMMA * mach ** 2))
    hmin = np.inf
    for m in meshes:
        X = m.xyz[m.elem_vert]
        pairs = ((0, 1), (0, 2), (1, 3), (2, 3)) if m.dim == 2 else ((0, 1), (0, 2), (0, 4))
        for a, b in pairs:
            hmin = min(hmin, np.linalg.norm(X[:, a] - X[:, b], axis=1).min())
    return cfl * hmin / ((1.0 + c) * (p + 1) ** 2)


def fp32_input(case: Case, u):
    """The state the mixed-precision path computes with for the FP64 state u
    (FP32 perturbation about the case's free stream)."""
    ur = S.reference_conserved(case.dim, 1.0, case.v_inf[:case.dim], case.p_inf, GAMMA)
    return S.fp32_perturbation_input(u, ur)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# --------------------------------------------------------------------------
# the workloads, small enough for the oracle
# --------------------------------------------------------------------------

def vortex_case(n=16, p=2, jitter=0.0):
    return Case("vortex", [M.vortex_mesh(n, jitter=jitter)], p, False, 0.0, 0.5, rk="rk4",
                dt=1e-3, v_inf=(0.5 * np.sqrt(GAMMA), 0.0), p_ref=1.0)


def periodic_ns_case(n=6, p=3, jitter=0.2):
    return Case("periodic_ns", [M.vortex_mesh(n, jitter=jitter, seed=3)], p, True, 0.02, 0.3,
                dt=2e-3)


def tgv_case(n=4, p=3):
    return Case("tgv", [M.tgv_mesh(n)], p, True, 1.0 / 1600.0, 0.1, dt=2e-3,
                v_inf=(0.0, 0.0, 0.0))


def cavity_case(target=1500, p=3):
    m = M.cavity_mesh(target)
    return Case("cavity", [m], p, True, 1.0 / 1500.0, 0.15, dt=cfl_dt([m], 0.15, p),
                inflow_delta=0.2, inflow_ywall=0.0)


def airfoil_case(n_inst=3, e_lo=300, e_hi=700, p=3, seed=7):
    ms = M.airfoil_batch(n_inst, seed=seed, e_lo=e_lo, e_hi=e_hi, p_geo=p)
    return Case("airfoil", ms, p, True, 1.0 / 23000.0, 0.2, dt=cfl_dt(ms, 0.2, p))


def tandem_case(n_inst=2, n_hex=1200, n_span=4, p=4, seed=7):
    """Tandem cylinders, 3-D hexes at p = 4, Re = 1000, M = 0.2."""
    import numpy as _np
    rng = _np.random.default_rng(seed)
    ms = [M.tandem_cylinders(rng.uniform(2.0, 5.0), rng.uniform(0.5, 1.5), n_hex, n_span, q=2)
          for _ in range(n_inst)]
    return Case("tandem", ms, p, True, 1.0 / 1000.0, 0.2, dt=cfl_dt(ms, 0.2, p),
                v_inf=(1.0, 0.0, 0.0))
