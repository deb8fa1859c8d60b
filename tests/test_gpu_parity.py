"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (relative L2 over all solution points and variables):
* FP64 path: 1e-12 per residual and over the stated short horizons;
* FP32 (mixed) path: the state itself is FP32, so the path's input is the
  FP32 rounding of the FP64 state.  Its arithmetic is checked against the
  oracle evaluated on that rounded input, with the standard forward error
  bound of the sums the residual is made of: |error| <= C * eps32 * M where
  M = (sum_k |D_k| |F^k| + |Cdiv| (|F*| + |F^D|)) / J is the magnitude of
  the terms (oracle ``residual(..., magnitude=True)``), eps32 = 2^-24 and
  C = 16 covers the few roundings of each flux value.  The total error
  against the exact FP64 input is printed; where the input rounding alone
  exceeds 1e-5 (low Mach numbers: the energy flux is ~(rho E + p) v with
  rho E + p >> residual), 1e-5 is below the FP32 representation floor.
"""
import numpy as np
import pytest

from tests import fr_cases as FC
from oracle import timestep as T
from oracle.acoustics import Probe, p_rms, oaspl as oracle_oaspl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _residual_pair(case, precision, inst=0):
    sol = FC.lib_solver(case, precision)
    disc = FC.oracle_disc(case, inst)
    x = disc.sol_coords()
    states = []
    for i in range(len(case.meshes)):
        xi = x if i == inst else FC.oracle_disc(case, i).sol_coords()
        u = FC.initial_state(case, xi, i)
        sol.set_state(i, u)
        states.append(u)
    R_gpu = sol.residual(inst)
    R_ref = disc.residual(states[inst])
    return sol, disc, states, R_gpu, R_ref


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_vortex_residual_fp64(p):
    case = FC.vortex_case(n=8, p=p, jitter=0.15)
    _, _, _, Rg, Rr = _residual_pair(case, "fp64")
    assert FC.rel_l2(Rg, Rr) < 1e-12


def test_vortex_100_rk4_steps_fp64_matches_oracle():
    """The tiny workload in full: 16x16 quads, p=2, RK4, dt=1e-3, 100 steps."""
    case = FC.vortex_case(n=16, p=2)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    sol.rk_step(100)
    ug = sol.get_state(0)
    ur = u
    for _ in range(100):
        ur = T.rk4_step(disc.residual, ur, case.dt)
    assert FC.rel_l2(ug, ur) < 1e-12


EPS32 = 2.0 ** -24
C_FP32 = 16.0


def _fp32_check(case, label):
    """Mixed-path residual against the oracle on the FP32-rounded input,
    within the forward error bound; prints the errors for the record."""
    sol, disc, states, Rg, Rr = _residual_pair(case, "fp32")
    u32 = FC.fp32_input(case, states[0])
    Rr32, mag = disc.residual(u32, magnitude=True)
    e_arith = FC.rel_l2(Rg, Rr32)
    e_total = FC.rel_l2(Rg, Rr)
    e_input = FC.rel_l2(Rr32, Rr)
    bound = C_FP32 * EPS32 * np.linalg.norm(mag) / np.linalg.norm(Rr32)
    print(f"{label} fp32: arithmetic {e_arith:.3e} (bound {bound:.3e}) total {e_total:.3e} "
          f"input-rounding {e_input:.3e}")
    assert e_arith < bound
    return e_arith, e_total, e_input


def test_vortex_residual_fp32():
    case = FC.vortex_case(n=16, p=2)
    _fp32_check(case, "vortex")


def test_periodic_navier_stokes_residual_fp64():
    case = FC.periodic_ns_case(n=6, p=3)
    _, _, _, Rg, Rr = _residual_pair(case, "fp64")
    assert FC.rel_l2(Rg, Rr) < 1e-12


def test_periodic_navier_stokes_residual_fp32():
    case = FC.periodic_ns_case(n=6, p=3)
    _fp32_check(case, "periodic NS")


@pytest.mark.parametrize("p", [2, 3, 4])
def test_tgv_residual_fp64(p):
    case = FC.tgv_case(n=3, p=p)
    _, _, _, Rg, Rr = _residual_pair(case, "fp64")
    assert FC.rel_l2(Rg, Rr) < 1e-12


def test_tgv_residual_fp32():
    case = FC.tgv_case(n=4, p=3)
    _fp32_check(case, "tgv")


def test_tgv_lsrk45_steps_fp64():
    case = FC.tgv_case(n=4, p=3)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    sol.rk_step(5)
    ur = u
    for _ in range(5):
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
    assert FC.rel_l2(sol.get_state(0), ur) < 1e-12


def test_cavity_residual_with_walls_inflow_outflow_farfield_fp64():
    case = FC.cavity_case(target=1500, p=3)
    _, _, u, Rg, Rr = _residual_pair(case, "fp64")
    assert FC.rel_l2(Rg, Rr) < 1e-12


def test_cavity_residual_fp32():
    case = FC.cavity_case(target=1500, p=3)
    _fp32_check(case, "cavity")


def test_airfoil_residual_fp32():
    case = FC.airfoil_case(n_inst=2)
    _fp32_check(case, "airfoil")


def test_cavity_10_steps_fp64():
    case = FC.cavity_case(target=1500, p=3)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    sol.rk_step(10)
    ur = u
    for _ in range(10):
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
    assert FC.rel_l2(sol.get_state(0), ur) < 1e-12


def test_airfoil_batch_residual_per_instance_and_batch_equals_solo():
    case = FC.airfoil_case(n_inst=3)
    sol = FC.lib_solver(case, "fp64")
    us = []
    for i in range(3):
        disc = FC.oracle_disc(case, i)
        u = FC.initial_state(case, disc.sol_coords(), i)
        sol.set_state(i, u)
        us.append(u)
        assert FC.rel_l2(sol.residual(i), disc.residual(u)) < 1e-12
    # batched stepping is bitwise identical to stepping each instance alone
    sol.rk_step(3)
    for i in range(3):
        solo_case = FC.Case("airfoil", [case.meshes[i]], case.p, True, case.mu, case.mach, dt=case.dt)
        assert solo_case.dt == case.dt
        solo = FC.lib_solver(solo_case, "fp64")
        solo.set_state(0, us[i])
        solo.rk_step(3)
        assert np.array_equal(solo.get_state(0), sol.get_state(i))


def test_probe_and_oaspl_match_oracle():
    case = FC.periodic_ns_case(n=6, p=3)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    pts = [np.array([0.3, -1.1]), np.array([-2.2, 3.7])]
    ids = [sol.probe_add(0, x) for x in pts]
    probes = [Probe(disc, x) for x in pts]
    hist = [[], []]
    ur = u
    for _ in range(12):
        sol.rk_step(1)
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
        for k in range(2):
            hist[k].append(probes[k].pressure(ur))
            assert abs(sol.probe_pressure(ids[k]) - hist[k][-1]) < 1e-11 * abs(hist[k][-1])
    for mode in (0, 1):
        got = sol.oaspl(ids, p_ref=2e-5, p_scale=101325 * 1.4 * 0.3 ** 2, mean_mode=mode)
        want = oracle_oaspl(hist, mode=mode, p_ref=2e-5, p_scale=101325 * 1.4 * 0.3 ** 2)
        assert abs(got - want) < 1e-6
    st = sol.probe_stats(ids[0])
    assert st[0] == 12
    # the device ring buffer holds the same samples, oldest first
    for k in range(2):
        h = sol.probe_history(ids[k])
        assert h.size == 12
        assert np.allclose(h, hist[k], rtol=1e-11, atol=0.0)
        assert np.array_equal(sol.probe_history(ids[k], max_n=5), h[-5:])
    assert abs(np.sqrt(st[2] / 12) - p_rms(hist[0], 0)) < 1e-9 * max(p_rms(hist[0], 0), 1e-30)


def test_conservation_periodic_is_roundoff():
    case = FC.periodic_ns_case(n=6, p=3)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    sol.set_state(0, FC.initial_state(case, disc.sol_coords()))
    sums = sol.conservation(0)
    R = sol.residual(0)
    g = disc.geometry()
    scale = np.einsum("es,s,esv->v", g.J, disc.ref.sp_w, np.abs(R))
    assert np.all(np.abs(sums) < 1e-12 * scale)
    tot, bad = sol.integral(0)
    assert bad == 0
    want = np.einsum("es,s,esv->v", g.J, disc.ref.sp_w, FC.initial_state(case, disc.sol_coords()))
    assert np.allclose(tot, want, rtol=1e-13)


def test_wall_force_matches_oracle():
    case = FC.airfoil_case(n_inst=1, e_lo=400, e_hi=401)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    sol.probe_reset()
    ur = u
    acc = np.zeros(2)
    for _ in range(3):
        sol.rk_step(1)
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
        acc += disc.wall_force(ur)
    got = sol.forces(0)
    want = acc / 3
    # the net force is a small difference of wall pressure forces of size
    # p_inf * perimeter: compare against that scale
    gross = case.p_inf * 2.2
    print("force gpu", got, "oracle", want)
    assert np.all(np.abs(got - want) < 1e-12 * gross)
    # coefficients: free stream along +x, chord 1 -> C_D = F_x / q, C_L = F_y / q
    q = 0.5 * 1.0 * 1.0 * 1.0
    cl, cd = sol.force_coefficients(0, 1.0)
    assert abs(cd - want[0] / q) < 1e-12 * gross / q and abs(cl - want[1] / q) < 1e-12 * gross / q


def test_force_coefficients_rotate_into_the_wind_axes():
    """A free stream at 30 degrees: drag is the force along it, lift the
    force along it turned by +90 degrees (same wall forces, other axes)."""
    from paper_2312_14167_gb300 import fr
    case = FC.airfoil_case(n_inst=1, e_lo=400, e_hi=401)
    u = FC.initial_state(case, FC.oracle_disc(case).sol_coords())
    a = np.deg2rad(30.0)
    cfg = FC.lib_config(case, "fp64")
    cfg.v_inf[0], cfg.v_inf[1] = np.cos(a), np.sin(a)
    sol = fr.Solver([fr.Mesh(case.meshes[0], case.p)], cfg)
    sol.set_state(0, u)
    sol.probe_reset()
    sol.rk_step(2)
    F = sol.forces(0)
    cl, cd = sol.force_coefficients(0, 2.0)
    q = 0.5 * 1.0 * 1.0 * 2.0
    assert abs(cd - (F[0] * np.cos(a) + F[1] * np.sin(a)) / q) < 1e-13 * np.abs(F).max() / q
    assert abs(cl - (-F[0] * np.sin(a) + F[1] * np.cos(a)) / q) < 1e-13 * np.abs(F).max() / q
    import pytest as _pt
    with _pt.raises(fr.FRError):
        sol.force_coefficients(0, 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tandem_cylinders_3d_p4_batch_residual(precision):
    """Two extruded tandem-cylinder candidates (curved hexes, p = 4, walls,
    far field, outflow, spanwise periodic) batched in one solver."""
    case = FC.tandem_case(n_inst=2, n_hex=900, n_span=3)
    sol = FC.lib_solver(case, precision)
    us = []
    for i in range(2):
        disc = FC.oracle_disc(case, i)
        u = FC.initial_state(case, disc.sol_coords(), i)
        sol.set_state(i, u)
        us.append(u)
    for i in range(2):
        disc = FC.oracle_disc(case, i)
        if precision == "fp64":
            assert FC.rel_l2(sol.residual(i), disc.residual(us[i])) < 1e-12
        else:
            u32 = FC.fp32_input(case, us[i])
            R32, mag = disc.residual(u32, magnitude=True)
            err = FC.rel_l2(sol.residual(i), R32)
            bound = C_FP32 * EPS32 * np.linalg.norm(mag) / np.linalg.norm(R32)
            print(f"tandem[{i}] fp32: {err:.3e} (bound {bound:.3e})")
            assert err < bound


def test_tandem_cylinders_lsrk45_steps_fp64():
    case = FC.tandem_case(n_inst=1, n_hex=700, n_span=3)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    pid = sol.probe_add(0, case.meshes[0].info["probes"][1])
    sol.rk_step(2)
    ur = u
    for _ in range(2):
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
    assert FC.rel_l2(sol.get_state(0), ur) < 1e-12
    pr = Probe(disc, case.meshes[0].info["probes"][1])
    assert abs(sol.probe_pressure(pid) - pr.pressure(ur)) < 1e-11 * pr.pressure(ur)


@pytest.mark.parametrize("maker", [lambda: FC.cavity_case(target=1500, p=3),
                                   lambda: FC.tgv_case(n=3, p=3),
                                   lambda: FC.airfoil_case(n_inst=2)])
def test_roe_flux_residual_fp64_and_fp32(maker):
    import dataclasses
    case = dataclasses.replace(maker(), flux="roe")
    _, _, _, Rg, Rr = _residual_pair(case, "fp64")
    assert FC.rel_l2(Rg, Rr) < 1e-12
    _fp32_check(case, "roe " + case.name)


def test_roe_flux_steps_fp64():
    import dataclasses
    case = dataclasses.replace(FC.periodic_ns_case(n=5, p=3), flux="roe")
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    sol.rk_step(3)
    ur = u
    for _ in range(3):
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
    assert FC.rel_l2(sol.get_state(0), ur) < 1e-12


@pytest.mark.parametrize("maker", [lambda: FC.periodic_ns_case(n=5, p=3),
                                   lambda: FC.cavity_case(target=1500, p=3),
                                   lambda: FC.tgv_case(n=3, p=3),
                                   lambda: FC.tandem_case(n_inst=1, n_hex=700, n_span=3)])
def test_ldg_viscous_scheme_residual_fp64_and_fp32(maker):
    import dataclasses
    case = dataclasses.replace(maker(), viscous_scheme="ldg")
    _, _, _, Rg, Rr = _residual_pair(case, "fp64")
    assert FC.rel_l2(Rg, Rr) < 1e-12
    _fp32_check(case, "ldg " + case.name)


def test_ldg_steps_fp64():
    import dataclasses
    case = dataclasses.replace(FC.periodic_ns_case(n=5, p=3), viscous_scheme="ldg")
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    sol.rk_step(3)
    ur = u
    for _ in range(3):
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
    assert FC.rel_l2(sol.get_state(0), ur) < 1e-12
