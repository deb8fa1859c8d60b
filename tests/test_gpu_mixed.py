"""Mixed precision (FP32 state, fluxes and contractions; FP64 geometry set-up
and FP64 observer sums) against the FP64 oracle:

* one residual per case, relative L2 against the oracle on the exact FP64
  input (the accuracy a user sees), at most 1e-5 where the input rounding
  of an FP32 state allows it (the FP32 state is stored as its perturbation
  about the free stream, so the input rounding is relative to that);
* stated short horizons: 100 RK4 steps of the isentropic vortex, 50 LSRK45
  steps of periodic Navier-Stokes, 10 LSRK45 steps of the cavity proxy; the
  state after the horizon (relative L2 below 1e-6 of the oracle's
  trajectory) and the residual evaluation there (within 1e-5 of the
  oracle's evaluation of the same state);
* OASPL (Sec. 3.1.2, Eqs. 9-12) from 240 samples of two observers in the
  periodic Navier-Stokes case, both mean readings, within 0.1 dB of the
  oracle.
"""
import numpy as np
import pytest

from tests import fr_cases as FC
from oracle import timestep as T
from oracle.acoustics import Probe, oaspl as oracle_oaspl

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = {
    "vortex": lambda: FC.vortex_case(n=8, p=3),
    "periodic_ns": lambda: FC.periodic_ns_case(n=6, p=3),
    "cavity": lambda: FC.cavity_case(target=1500, p=3),
    "airfoil": lambda: FC.airfoil_case(n_inst=1, e_lo=600, e_hi=700),
    "tandem": lambda: FC.tandem_case(n_inst=1, n_hex=900, n_span=3),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_residual_within_1e5_of_the_oracle(name):
    case = CASES[name]()
    sol = FC.lib_solver(case, "fp32")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    R = disc.residual(u)
    err = FC.rel_l2(sol.residual(0), R)
    floor = FC.rel_l2(disc.residual(FC.fp32_input(case, u)), R)
    print(f"{name} fp32 residual vs oracle: {err:.3e} (input rounding alone {floor:.3e})")
    assert err < TOL_MIXED


def _horizon(case, steps, step_fn):
    """After the horizon: the state's relative L2 error against the oracle's
    trajectory; the residual evaluation there against the oracle's
    evaluation of the same state (the FP64 image of the FP32 state the
    solver holds); and, for the record, the residual against the oracle's
    residual on its own trajectory and the relative error of the state's
    change (both carry the rounding of the stored FP32 state, which the
    residual's derivatives amplify on thin wall cells)."""
    sol = FC.lib_solver(case, "fp32")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    sol.rk_step(steps)
    ug = sol.get_state(0)
    Rg = sol.residual(0)
    ur = u
    for _ in range(steps):
        ur = step_fn(disc.residual, ur, case.dt)
    return (FC.rel_l2(ug, ur), FC.rel_l2(Rg, disc.residual(ug)), FC.rel_l2(Rg, disc.residual(ur)),
            FC.rel_l2(ug - u, ur - u))


@pytest.mark.parametrize("name,steps,rk", [("vortex", 100, "rk4"), ("periodic_ns", 50, "lsrk45"),
                                           ("cavity", 10, "lsrk45")])
def test_mixed_horizon_matches_the_oracle(name, steps, rk):
    case = CASES[name]()
    assert case.rk == rk
    step_fn = T.rk4_step if rk == "rk4" else T.lsrk45_step
    state, resid, drift, change = _horizon(case, steps, step_fn)
    print(f"{name} fp32, {steps} {rk} steps: state {state:.3e}, residual evaluation at the end "
          f"{resid:.3e}, vs the oracle's trajectory {drift:.3e}, change of the state {change:.3e}")
    assert state < 1e-6 and resid < TOL_MIXED


def test_mixed_oaspl_within_a_tenth_of_a_decibel_on_the_periodic_case():
    case = FC.periodic_ns_case(n=6, p=3)
    sol = FC.lib_solver(case, "fp32")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    pts = [np.array([0.3, -1.1]), np.array([-2.2, 3.7])]
    ids = [sol.probe_add(0, x) for x in pts]
    probes = [Probe(disc, x) for x in pts]
    n = 240
    sol.rk_step(n)
    hist = [[], []]
    ur = u
    for _ in range(n):
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
        for k in range(2):
            hist[k].append(probes[k].pressure(ur))
    scale = 101325 * 1.4 * 0.3 ** 2
    for mode in (0, 1):
        got = sol.oaspl(ids, p_ref=2e-5, p_scale=scale, mean_mode=mode)
        want = oracle_oaspl(hist, mode=mode, p_ref=2e-5, p_scale=scale)
        print(f"mixed OASPL mode {mode}: {got:.6f} dB, oracle {want:.6f} dB, diff {got - want:.2e} dB")
        assert abs(got - want) < 0.1
    for k in range(2):
        h = sol.probe_history(ids[k])
        assert h.size == n and np.max(np.abs(h - hist[k])) < 1e-5 * np.max(np.abs(hist[k]))
