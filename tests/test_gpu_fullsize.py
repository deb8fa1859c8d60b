"""GPU parity at the full sizes of the workloads, on sampled outputs the
oracle computes element by element (its residual restricted to a subset
evaluates only their two-ring neighbourhood), and through properties that
hold at any size.

* cavity proxy, ~32k quads, p = 3 (walls, tanh inflow, outflow, far field);
* Taylor-Green, 16^3 hexes p = 3 against the oracle; 64^3 hexes p = 3 (16.8 M
  solution points, the oracle cannot afford it) through the exact kinetic
  energy rate of the divergence-free initial field,
  dE_k/dt = -nu <|omega|^2> Vol = -(3/4) nu (2 pi)^3, and conservation;
* the 32-candidate NACA poll (849k curved quads) as the bench runs it.
Tolerances: FP64 1e-12, or the FP64 forward error bound 16 eps64 sum|terms|
where that is larger (a low-Mach residual is a 1e-4 fraction of its flux
terms, so two correct FP64 evaluations in different summation orders may
differ by more than 1e-12); FP32 the forward error bound 16 eps32 sum|terms|.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from tests import fr_cases as FC
from synth import meshes as M, states as S
from oracle import timestep as T

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -53


def _fp64_tol(disc, u, elems=None):
    _, mag = disc.residual(u, elems, magnitude=True)
    R = disc.residual(u, elems)
    return max(1e-12, 16 * EPS64 * np.linalg.norm(mag) / np.linalg.norm(R))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sample(mesh, n, seed, disc):
    rng = np.random.default_rng(seed)
    el = rng.choice(mesh.n_elem, size=min(n, mesh.n_elem), replace=False)
    bnd = np.nonzero(np.any(disc.bc > 0, axis=1))[0]
    if bnd.size:
        el = np.union1d(el, rng.choice(bnd, size=min(16, bnd.size), replace=False))
    return np.unique(el)


def _check_sampled(case, inst, sol_by_prec, us):
    disc = FC.oracle_disc(case, inst)
    el = _sample(case.meshes[inst], 48, inst, disc)
    u = us[inst]
    R64 = disc.residual(u, el)
    if "fp64" in sol_by_prec:
        Rg = sol_by_prec["fp64"].residual(inst)[el]
        tol = _fp64_tol(disc, u, el)
        print(f"{case.name}[{inst}] fp64 sampled: {FC.rel_l2(Rg, R64):.3e} (tol {tol:.3e})")
        assert FC.rel_l2(Rg, R64) < tol
    if "fp32" in sol_by_prec:
        u32 = FC.fp32_input(case, u)
        R32, mag = disc.residual(u32, el, magnitude=True)
        Rg = sol_by_prec["fp32"].residual(inst)[el]
        err = FC.rel_l2(Rg, R32)
        bound = 16 * EPS32 * np.linalg.norm(mag) / np.linalg.norm(R32)
        print(f"{case.name}[{inst}] fp32 sampled: {err:.3e} (bound {bound:.3e}), "
              f"total {FC.rel_l2(Rg, R64):.3e}")
        assert err < bound


def test_cavity_full_size_sampled_parity():
    case = FC.cavity_case(target=32000, p=3)
    assert 30000 < case.meshes[0].n_elem < 34000
    sols = {p: FC.lib_solver(case, p) for p in ("fp64", "fp32")}
    x = sols["fp64"].meshes[0].sol_coords()
    u = FC.initial_state(case, x)
    for s in sols.values():
        s.set_state(0, u)
    _check_sampled(case, 0, sols, [u])
    sols["fp32"].rk_step(5)
    _, bad = sols["fp32"].integral(0)
    assert bad == 0


def test_tgv_16_fp64_matches_oracle_residual_and_step():
    case = FC.tgv_case(n=16, p=3)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    tol = _fp64_tol(disc, u)
    err = FC.rel_l2(sol.residual(0), disc.residual(u))
    print(f"tgv16 fp64 residual: {err:.3e} (tol {tol:.3e})")
    assert err < tol
    sol.rk_step(1)
    assert FC.rel_l2(sol.get_state(0), T.lsrk45_step(disc.residual, u, case.dt)) < 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-3)])
def test_tgv_64_kinetic_energy_rate_and_conservation(precision, tol):
    n = 64
    case = FC.tgv_case(n=n, p=3)
    sol = FC.lib_solver(case, precision)
    x = sol.meshes[0].sol_coords()
    u = S.taylor_green(x, mach=0.1)
    sol.set_state(0, u)
    R = sol.residual(0)
    # affine box: J = (h/2)^3 at every point; tensor Gauss weights
    h = 2 * np.pi / n
    _, w1 = npleg.leggauss(4)
    w = np.einsum("i,j,k->kji", w1, w1, w1).ravel()        # xi fastest
    rho = u[..., 0]
    v = u[..., 1:4] / rho[..., None]
    dek = np.einsum("esi,esi->es", v, R[..., 1:4]) - 0.5 * np.sum(v * v, -1) * R[..., 0]
    rate = (h / 2) ** 3 * np.einsum("s,es->", w, dek)
    expected = -0.75 / 1600.0 * (2 * np.pi) ** 3
    print(f"tgv64 {precision}: dE_k/dt = {rate:.8e}, analytic {expected:.8e}")
    assert abs(rate / expected - 1.0) < tol
    sums = sol.conservation(0)
    scale = (h / 2) ** 3 * np.einsum("s,esv->v", w, np.abs(R))
    assert np.all(np.abs(sums) < (1e-10 if precision == "fp64" else 1e-4) * scale)


def test_airfoil_poll_full_size_sampled_parity():
    meshes = M.airfoil_batch(32, seed=2312)
    case = FC.Case("airfoil", meshes, 3, True, 1.0 / 23000.0, 0.2,
                   dt=FC.cfl_dt(meshes, 0.2, 3))
    sols = {p: FC.lib_solver(case, p) for p in ("fp64", "fp32")}
    us = []
    for i, m in enumerate(sols["fp64"].meshes):
        u = FC.initial_state(case, m.sol_coords(), i)
        us.append(u)
        for s in sols.values():
            s.set_state(i, u)
    for inst in (0, 17, 31):
        _check_sampled(case, inst, sols, us)


def test_tandem_candidate_full_size_sampled_parity():
    """One tandem-cylinder candidate at the top of the poll's size range
    (about 150k curved hexes, p = 4: 18.75 M solution points)."""
    m = M.tandem_cylinders(3.1, 1.3, 150000, 16, q=2)
    assert 120000 < m.n_elem < 170000
    case = FC.Case("tandem", [m], 4, True, 1.0 / 1000.0, 0.2, dt=FC.cfl_dt([m], 0.2, 4),
                   v_inf=(1.0, 0.0, 0.0))
    sols = {p: FC.lib_solver(case, p) for p in ("fp64", "fp32")}
    u = FC.initial_state(case, sols["fp64"].meshes[0].sol_coords())
    for s in sols.values():
        s.set_state(0, u)
    _check_sampled(case, 0, sols, [u])
    sols["fp32"].rk_step(3)
    _, bad = sols["fp32"].integral(0)
    assert bad == 0


def test_airfoil_sponge_candidate_full_size_parity():
    """The smallest candidate of the variable-degree airfoil poll (about 8k
    curved quads; p = 3 within 4 chords, 2 to 8, 1 to 12, 0 beyond): the
    whole residual against the variable-degree oracle, FP64 and FP32."""
    from oracle.fr_var import VarFRDiscretisation
    from oracle.physics import NavierStokes
    from paper_2312_14167_gb300 import fr
    meshes = M.airfoil_batch(32, seed=2312)
    m = min(meshes, key=lambda mm: mm.n_elem)
    ep = M.sponge_degrees(m, (0.5, 0.0), (4.0, 8.0, 12.0), (3, 2, 1, 0))
    assert set(np.unique(ep)) == {0, 1, 2, 3}
    case = FC.Case("airfoil", [m], 3, True, 1.0 / 23000.0, 0.2, dt=FC.cfl_dt([m], 0.2, 3))
    ph = NavierStokes(2, gamma=FC.GAMMA, mu=case.mu, prandtl=FC.PR, viscous=True, rho_inf=1.0,
                      v_inf=case.v_inf, p_inf=case.p_inf)
    d = VarFRDiscretisation(m, ep, ph)
    u = FC.initial_state(case, d.sol_coords())
    R, mag = d.residual(u, magnitude=True)
    s64 = fr.Solver([fr.Mesh(m, ep)], FC.lib_config(case, "fp64"))
    s64.set_state(0, u)
    tol = max(1e-12, 16 * EPS64 * np.linalg.norm(mag) / np.linalg.norm(R))
    err = FC.rel_l2(s64.residual(0), R)
    print(f"sponge candidate fp64: {err:.3e} (tol {tol:.3e})")
    assert err < tol
    s32 = fr.Solver([fr.Mesh(m, ep)], FC.lib_config(case, "fp32"))
    s32.set_state(0, u)
    u32 = FC.fp32_input(case, u)
    R32, mag32 = d.residual(u32, magnitude=True)
    err32 = FC.rel_l2(s32.residual(0), R32)
    bound = 16 * EPS32 * np.linalg.norm(mag32) / np.linalg.norm(R32)
    print(f"sponge candidate fp32: {err32:.3e} (bound {bound:.3e})")
    assert err32 < bound
