"""GPU parity of the variable-degree path (a polynomial degree per element,
mortar coupling of the faces joining two degrees) against the oracle
``oracle.fr_var``: residual and RK steps in FP64 (1e-12), FP32 within its
forward error bound, conservation, probes and wall forces in degree groups,
a batch mixing variable-degree and uniform meshes of different degrees, and
the host reordering of the state (element order <-> degree groups)."""
import numpy as np
import pytest

from synth import meshes as M, states as S
from oracle.fr_var import VarFRDiscretisation
from oracle.physics import NavierStokes
from oracle import timestep as T
from tests.fr_cases import cfl_dt

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -53
GAMMA, PR, MACH, MU = 1.4, 0.71, 0.3, 0.01


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _box(dim, seed=5, degrees=(1, 2, 3, 4)):
    n = (6, 5) if dim == 2 else (3, 3, 2)
    m = M.reorient(M.periodic_box(dim, n, (0.0,) * dim, (1.0,) * dim, jitter=0.2), seed)
    return m, M.checker_degrees(m, degrees, seed=seed)


def _cavity():
    m = M.cavity_mesh(600)
    return m, M.sponge_degrees(m, (0.25, 0.0), (1.5, 4.0), (3, 2, 1))


def _airfoil():
    m = M.naca_omesh(0.04, 0.4, 0.12, 4.0, 600)
    return m, M.sponge_degrees(m, (0.5, 0.0), (2.0, 6.0), (4, 3, 2))


def _tandem():
    """Curved (q = 2) tandem-cylinder hexes: O-rings and the Cartesian
    background meet in non-trivial face orientations; 564 faces join two
    degrees."""
    m = M.tandem_cylinders(2.5, 0.8, 900, 3)
    return m, M.sponge_degrees(m, (1.25, 0.0), (2.5, 5.0), (3, 2, 1))


MESHES = {"box2d": lambda: _box(2), "box3d": lambda: _box(3), "cavity": _cavity,
          "airfoil": _airfoil,
          # with degree-0 (one-point, finite-volume) elements
          "box2d0": lambda: _box(2, degrees=(0, 1, 2, 3)),
          "box3d0": lambda: _box(3, degrees=(0, 1, 2, 3)),
          "tandem": _tandem}


# viscosity per case: the airfoil grids have 1e-3-thick wall cells, where
# mu = 0.01 would put the explicit viscous step limit far below the CFL step;
# they run at the airfoil workload's Re_c = 23000
MU_CASE = {"airfoil": 1.0 / 23000.0, "tandem": 1.0e-3}


def _phys(dim, viscous, flux, mu=MU):
    return NavierStokes(dim, gamma=GAMMA, mu=mu if viscous else 0.0, prandtl=PR, viscous=viscous,
                        rho_inf=1.0, v_inf=(1.0, 0.0, 0.0)[:dim], p_inf=1.0 / (GAMMA * MACH ** 2),
                        flux=flux)


def _solver(meshes_eps, viscous, scheme, flux, precision, rk="lsrk45", dt=1e-4, mu=MU):
    from paper_2312_14167_gb300 import fr
    dim = meshes_eps[0][0].dim
    cfg = fr.make_config(dim, gamma=GAMMA, prandtl=PR, mu=mu if viscous else 0.0, rho_inf=1.0,
                         v_inf=(1.0, 0.0, 0.0)[:dim], p_inf=1.0 / (GAMMA * MACH ** 2), dt=dt,
                         viscous=viscous, rk=fr.FR_RK4 if rk == "rk4" else fr.FR_LSRK45,
                         precision=fr.FR_FP64 if precision == "fp64" else fr.FR_FP32,
                         flux=fr.FR_FLUX_ROE if flux == "roe" else fr.FR_FLUX_RUSANOV,
                         viscous_scheme=fr.FR_VISC_LDG if scheme == "ldg" else fr.FR_VISC_BR2)
    return fr.Solver([fr.Mesh(m, ep) for m, ep in meshes_eps], cfg)


def _dt(m, ep):
    """Fixed step within the CFL limit of the finest, highest-degree elements."""
    return min(1e-4, cfl_dt([m], MACH, int(np.max(ep))))


def _state(x, dim, seed=3, mesh=None):
    u = S.smooth_perturbed(x, dim, MACH, amp=0.05, seed=seed)
    if mesh is not None and "wall_points" in mesh.info:
        u = S.wall_damped(x, mesh.info["wall_points"], 0.05, u)
    return u


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [("box2d", False, "br2", "rusanov"), ("box2d", True, "br2", "rusanov"),
         ("box2d", True, "ldg", "rusanov"), ("box2d", True, "br2", "roe"),
         ("box3d", False, "br2", "rusanov"), ("box3d", True, "br2", "rusanov"),
         ("box3d", True, "ldg", "roe"), ("cavity", True, "br2", "rusanov"),
         ("cavity", True, "ldg", "rusanov"), ("airfoil", True, "br2", "rusanov"),
         ("box2d0", False, "br2", "rusanov"), ("box2d0", True, "br2", "rusanov"),
         ("box2d0", True, "ldg", "roe"), ("box3d0", False, "br2", "rusanov"),
         ("box3d0", True, "br2", "rusanov"), ("box3d0", True, "ldg", "rusanov"),
         ("tandem", True, "br2", "rusanov"), ("tandem", True, "ldg", "roe")]


@pytest.mark.parametrize("name,viscous,scheme,flux", CASES)
def test_fp64_residual_and_steps_match_oracle(name, viscous, scheme, flux):
    m, ep = MESHES[name]()
    dim = m.dim
    mu = MU_CASE.get(name, MU)
    d = VarFRDiscretisation(m, ep, _phys(dim, viscous, flux, mu), viscous_scheme=scheme)
    dt = _dt(m, ep)
    sol = _solver([(m, ep)], viscous, scheme, flux, "fp64", dt=dt, mu=mu)
    x = sol.meshes[0].sol_coords()
    assert np.abs(x - d.sol_coords()).max() < 1e-12
    u = _state(x, dim, mesh=m)
    sol.set_state(0, u)
    assert np.array_equal(sol.get_state(0), u)
    R = d.residual(u)
    err = _rel(sol.residual(0), R)
    print(f"{name} visc={viscous} {scheme} {flux}: fp64 residual {err:.3e}")
    assert err < 1e-12
    sol.rk_step(3)
    ur = u
    for _ in range(3):
        ur = T.lsrk45_step(d.residual, ur, dt)
    assert _rel(sol.get_state(0), ur) < 1e-12


def test_rk4_steps_match_oracle():
    m, ep = _box(2, seed=8)
    d = VarFRDiscretisation(m, ep, _phys(2, True, "rusanov"))
    sol = _solver([(m, ep)], True, "br2", "rusanov", "fp64", rk="rk4")
    u = _state(sol.meshes[0].sol_coords(), 2, seed=9)
    sol.set_state(0, u)
    sol.rk_step(2)
    ur = u
    for _ in range(2):
        ur = T.rk4_step(d.residual, ur, 1e-4)
    assert _rel(sol.get_state(0), ur) < 1e-12


@pytest.mark.parametrize("name,scheme", [("box2d", "br2"), ("box3d", "ldg"), ("cavity", "br2"),
                                         ("box2d0", "ldg"), ("box3d0", "br2"), ("tandem", "br2")])
def test_fp32_residual_within_forward_error_bound(name, scheme):
    m, ep = MESHES[name]()
    mu = MU_CASE.get(name, MU)
    d = VarFRDiscretisation(m, ep, _phys(m.dim, True, "rusanov", mu), viscous_scheme=scheme)
    sol = _solver([(m, ep)], True, scheme, "rusanov", "fp32", mu=mu)
    u = _state(sol.meshes[0].sol_coords(), m.dim, mesh=m)
    sol.set_state(0, u)
    u32 = S.fp32_perturbation_input(u, S.reference_conserved(m.dim, 1.0, (1.0, 0.0, 0.0), 1.0 / (GAMMA * MACH ** 2), GAMMA))
    R, mag = d.residual(u32, magnitude=True)
    err = _rel(sol.residual(0), R)
    bound = 16 * EPS32 * np.linalg.norm(mag) / np.linalg.norm(R)
    print(f"{name} fp32: {err:.3e} (bound {bound:.3e})")
    assert err < bound


@pytest.mark.parametrize("dim", [2, 3])
def test_mixed_degree_conservation_on_gpu(dim):
    m, ep = _box(dim)
    sol = _solver([(m, ep)], True, "br2", "rusanov", "fp64")
    d = VarFRDiscretisation(m, ep, _phys(dim, True, "rusanov"))
    u = _state(sol.meshes[0].sol_coords(), dim)
    sol.set_state(0, u)
    sums = sol.conservation(0)
    scale = d.integral(np.abs(d.residual(u)))
    assert np.all(np.abs(sums) < 1e-12 * scale.max())
    # the integral of the state through both reductions
    ref = d.integral(u)
    got, bad = sol.integral(0)
    got_s, bad_s = sol.integral_static(0)
    assert bad == 0 and bad_s == 0
    assert np.allclose(got, ref, rtol=1e-13) and np.allclose(got_s, ref, rtol=1e-13)


def test_probes_and_wall_force_in_degree_groups():
    m, ep = _airfoil()
    mu = MU_CASE["airfoil"]
    d = VarFRDiscretisation(m, ep, _phys(2, True, "rusanov", mu))
    dt = _dt(m, ep)
    sol = _solver([(m, ep)], True, "br2", "rusanov", "fp64", dt=dt, mu=mu)
    x = sol.meshes[0].sol_coords()
    u = _state(x, 2, mesh=m)
    sol.set_state(0, u)
    # one observer near the wall (degree 4), one in the outer sponge (degree 2)
    pts = [np.array([1.0, -0.3]), np.array([0.0, 9.0])]
    ids = [sol.probe_add(0, p) for p in pts]
    sol.probe_reset()
    sol.rk_step(1)
    un = sol.get_state(0)
    ref_u = T.lsrk45_step(d.residual, u, dt)
    assert _rel(un, ref_u) < 1e-12
    for pid, p in zip(ids, pts):
        ps = d.phys.pressure(d.probe_state(ref_u, p)[None, :])[0]
        assert abs(sol.probe_pressure(pid) - ps) < 1e-12 * abs(ps)
    F = sol.forces(0)
    Fr = d.wall_force(ref_u)
    assert np.allclose(F, Fr, rtol=1e-10, atol=1e-12 * np.abs(Fr).max())


def test_batch_of_variable_and_uniform_meshes_of_several_degrees():
    """Three instances: two variable-degree boxes and a uniform degree-2
    vortex mesh; each instance's residual and two steps match the oracle."""
    a, ea = _box(2, seed=5)
    b, eb = _box(2, seed=11)
    c = M.vortex_mesh(4, jitter=0.1)
    ec = np.full(c.n_elem, 2, dtype=np.int32)
    sol = _solver([(a, ea), (b, eb), (c, 2)], True, "br2", "rusanov", "fp64")
    discs = [VarFRDiscretisation(mm, ee, _phys(2, True, "rusanov")) for mm, ee in ((a, ea), (b, eb), (c, ec))]
    us = []
    for i, d in enumerate(discs):
        x = sol.meshes[i].sol_coords().reshape(-1, 2)
        u = _state(x, 2, seed=20 + i)
        sol.set_state(i, u.reshape(sol.meshes[i].state_shape + (4,)))
        us.append(u)
    for i, d in enumerate(discs):
        assert _rel(sol.residual(i).reshape(-1, 4), d.residual(us[i])) < 1e-12
    sol.rk_step(2)
    for i, d in enumerate(discs):
        ur = us[i]
        for _ in range(2):
            ur = T.lsrk45_step(d.residual, ur, 1e-4)
        assert _rel(sol.get_state(i).reshape(-1, 4), ur) < 1e-12
    # all instances in one call each way: the same values as one call per instance
    flat = sol.get_states()
    assert np.array_equal(flat, np.concatenate([sol.get_state(i).reshape(-1) for i in range(3)]))
    new = np.concatenate([(u * 1.01).reshape(-1) for u in us])
    sol.set_states(new)
    off = 0
    for i, u in enumerate(us):
        assert np.array_equal(sol.get_state(i).reshape(-1), new[off:off + u.size])
        off += u.size
    sol.set_state(1, us[1].reshape(sol.meshes[1].state_shape + (4,)))
    assert np.array_equal(sol.get_states()[us[0].size:us[0].size + us[1].size], us[1].reshape(-1))
    with pytest.raises(ValueError):
        sol.set_states(new[:-1])
    # determinism: a candidate advanced inside the batch (degree groups and
    # mortar passes shared with the others) is bitwise the candidate alone
    solo = _solver([(b, eb)], True, "br2", "rusanov", "fp64")
    u1 = us[1].reshape(sol.meshes[1].state_shape + (4,))
    solo.set_state(0, u1)
    sol.set_states(np.concatenate([u.reshape(-1) for u in us]))
    solo.rk_step(2)
    sol.rk_step(2)
    assert np.array_equal(solo.get_state(0), sol.get_state(1))
    assert np.array_equal(solo.residual(0), sol.residual(1))
