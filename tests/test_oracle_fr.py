"""Pins of the oracle's FR residual (Sec. 2.3) and Navier-Stokes physics
(Sec. 2.1, Eqs. 1-7) against properties fixed by the mathematics:

* free-stream preservation on jittered, trilinear and curved meshes;
* conservation to round-off on periodic meshes and closed walled boxes;
* equivalence with a separately written strong-form nodal DG-SEM on
  affine meshes (the DG-recovery correction reproduces nodal DG);
* design-order convergence on the exact isentropic vortex;
* heat-equation decay through the gradient / BR2 / viscous-flux path;
* closed-form instantaneous viscous residuals of a shear wave and of a
  resting temperature field (they fix the signs of the viscous work and the
  heat flux: viscous dissipation must heat the fluid, heat flows from hot to
  cold);
* Rusanov consistency and skew symmetry; wall and far-field boundary states;
* a closed body under uniform pressure feels no net force.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from synth import meshes as M, states as S
from oracle.fr import FRDiscretisation
from oracle.physics import NavierStokes, ScalarDiffusion
from oracle import timestep as T
from oracle.acoustics import Probe


def _fs_max(disc, mach=0.3, direction=(1.0, 0.4)):
    x = disc.sol_coords()
    U = S.free_stream(x.shape[:-1], disc.mesh.dim, mach, direction=direction)
    R = disc.residual(U)
    return np.abs(R).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("visc", [False, True])
def test_free_stream_preserved_jittered_quads(p, visc):
    m = M.vortex_mesh(5, jitter=0.25, seed=p)
    d = FRDiscretisation(m, p, NavierStokes(2, mu=0.02, viscous=visc))
    assert _fs_max(d) < 1e-11


@pytest.mark.parametrize("p", [2, 3])
def test_free_stream_preserved_jittered_trilinear_hexes(p):
    m = M.periodic_box(3, (3, 3, 3), (0, 0, 0), (1, 1.3, 0.9), jitter=0.2, seed=5)
    d = FRDiscretisation(m, p, NavierStokes(3, mu=0.01, viscous=True))
    assert _fs_max(d, direction=(1.0, 0.3, -0.2)) < 1e-10


def test_free_stream_preserved_curved_omesh_with_farfield():
    m = M.naca_omesh(0.04, 0.4, 0.12, 3.0, 600, p_geo=3)
    ph = NavierStokes(2, viscous=False, rho_inf=1.0, v_inf=(1.0, 0.0),
                      p_inf=1.0 / (1.4 * 0.2 ** 2))
    d = FRDiscretisation(m, 3, ph)
    # tangential-only flow is not uniform at the wall; test the far ring only
    x = d.sol_coords()
    U = S.free_stream(x.shape[:-1], 2, 0.2)
    R = d.residual(U)
    far = np.nonzero(np.all(d.bc != 2, axis=1))[0]
    nbr_wall = np.unique(d.partner_elem[np.any(d.bc == 2, axis=1)])
    far = np.setdiff1d(far, nbr_wall)
    # round-off relative to each element's flux scale p_inf |S| / J
    g = d.geometry()
    scale = (1.0 / (1.4 * 0.04)) * np.abs(g.S).max(axis=(1, 2, 3)) / g.J.min(axis=1)
    assert np.all(np.abs(R[far]).max(axis=(1, 2)) < 1e-11 * scale[far])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_conservation_periodic_navier_stokes(p):
    m = M.vortex_mesh(4, jitter=0.2)
    d = FRDiscretisation(m, p, NavierStokes(2, mu=0.05, viscous=True))
    g = d.geometry()
    U = S.random_state(m.n_elem, d.ref.nsp, 2, 0.3, amp=0.1)
    R = d.residual(U)
    tot = np.einsum("es,s,esv->v", g.J, d.ref.sp_w, R)
    scale = np.einsum("es,s,esv->v", g.J, d.ref.sp_w, np.abs(R))
    assert np.all(np.abs(tot) < 1e-13 * scale)


def test_closed_walled_box_conserves_mass_and_energy():
    m = M.periodic_box(2, (4, 3), (0, 0), (2, 1.5), jitter=0.15)
    m.face_tag[m.face_tag == M.TAG_PERIODIC] = M.TAG_WALL
    d = FRDiscretisation(m, 3, NavierStokes(2, mu=0.03, viscous=True))
    g = d.geometry()
    U = S.random_state(m.n_elem, d.ref.nsp, 2, 0.3, amp=0.1)
    R = d.residual(U)
    tot = np.einsum("es,s,esv->v", g.J, d.ref.sp_w, R)
    scale = np.einsum("es,s,esv->v", g.J, d.ref.sp_w, np.abs(R))
    assert abs(tot[0]) < 1e-13 * scale[0]
    assert abs(tot[-1]) < 1e-13 * scale[-1]


def _dgsem_euler_residual(U, nx, ny, lo, hi, p, phys):
    """Strong-form nodal DG spectral-element residual on a periodic Cartesian
    grid, written element by element and line by line with library Gauss
    nodes; surface terms lifted with l_i(+-1)/w_i."""
    xg, wg = npleg.leggauss(p + 1)
    n = p + 1
    V = np.vander(xg, n, increasing=True)
    coef = np.linalg.inv(V)                          # monomial coefficients of l_j
    def lag(t):
        return np.vander(np.atleast_1d(t), n, increasing=True) @ coef
    dcoef = np.array([np.polynomial.polynomial.polyder(coef[:, j]) for j in range(n)]).T
    def dlag(t):
        if n == 1:
            return np.zeros((np.size(t), 1))
        return np.vander(np.atleast_1d(t), n - 1, increasing=True) @ dcoef
    Dm = dlag(xg)
    lm, lp = lag(-1.0)[0], lag(1.0)[0]
    dx = (hi[0] - lo[0]) / nx
    dy = (hi[1] - lo[1]) / ny
    nv = U.shape[-1]
    Ue = U.reshape(ny, nx, n, n, nv)                 # [j_elem, i_elem, eta, xi, v]
    out = np.zeros_like(Ue)
    for axis, h, (cnt, ) in ((0, dx, (nx,)), (1, dy, (ny,))):
        nvec = np.zeros(2)
        nvec[axis] = 1.0
        for je in range(ny):
            for ie in range(nx):
                for line in range(n):
                    if axis == 0:
                        u = Ue[je, ie, line, :, :]
                        nb = Ue[je, (ie + 1) % nx, line, :, :]
                        nbm = Ue[je, (ie - 1) % nx, line, :, :]
                    else:
                        u = Ue[je, ie, :, line, :]
                        nb = Ue[(je + 1) % ny, ie, :, line, :]
                        nbm = Ue[(je - 1) % ny, ie, :, line, :]
                    f = phys.inviscid_flux(u)[:, axis, :]
                    fp = lp @ f
                    fm = lm @ f
                    up, um = lp @ u, lm @ u
                    fs_r = phys.rusanov(up[None], (lm @ nb)[None], nvec[None])[0]
                    fs_l = phys.rusanov((lp @ nbm)[None], um[None], nvec[None])[0]
                    r = Dm @ f + np.outer(lp / wg, fs_r - fp) - np.outer(lm / wg, fs_l - fm)
                    r *= -2.0 / h
                    if axis == 0:
                        out[je, ie, line, :, :] += r
                    else:
                        out[je, ie, :, line, :] += r
    return out.reshape(U.shape)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_fr_dg_recovery_equals_nodal_dgsem_on_affine_meshes(p):
    for nx, ny in ((1, 1), (2, 3), (3, 2)):
        lo, hi = (-1.0, -0.5), (1.5, 1.0)
        m = M.periodic_box(2, (nx, ny), lo, hi)
        ph = NavierStokes(2)
        d = FRDiscretisation(m, p, ph)
        x = d.sol_coords()
        U = S.smooth_perturbed(x, 2, 0.4, amp=0.2, seed=p)
        R_fr = d.residual(U)
        R_dg = _dgsem_euler_residual(U, nx, ny, lo, hi, p, ph)
        scale = np.abs(R_fr).max()
        assert np.abs(R_fr - R_dg).max() < 1e-13 * max(scale, 1.0)


def _vortex_error(n, p, steps=20, dt=5e-3):
    m = M.vortex_mesh(n)
    d = FRDiscretisation(m, p, NavierStokes(2))
    x = d.sol_coords()
    U = S.isentropic_vortex(x)
    for _ in range(steps):
        U = T.rk4_step(d.residual, U, dt)
    ex = S.isentropic_vortex(x, t=steps * dt)
    g = d.geometry()
    return np.sqrt(np.einsum("es,s,es->", g.J, d.ref.sp_w, (U - ex)[..., 0] ** 2))


@pytest.mark.slow
@pytest.mark.parametrize("p,min_order", [(2, 2.4), (3, 3.6)])
def test_isentropic_vortex_converges_at_design_order(p, min_order):
    e1, e2 = _vortex_error(16, p), _vortex_error(32, p)
    assert np.log2(e1 / e2) > min_order


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2, 3])
def test_heat_equation_decay_through_br2(p):
    nu = 0.1
    errs = []
    t_end, steps = 1.0, 400
    for n in (4, 8):
        two_pi = 2 * np.pi
        m = M.periodic_box(2, (n, n), (0, 0), (two_pi, two_pi))
        d = FRDiscretisation(m, p, ScalarDiffusion(2, nu))
        x = d.sol_coords()
        U = (np.sin(x[..., 0]) * np.sin(x[..., 1]))[..., None]
        for _ in range(steps):
            U = T.rk4_step(d.residual, U, t_end / steps)
        ex = np.exp(-2 * nu * t_end) * np.sin(x[..., 0]) * np.sin(x[..., 1])
        g = d.geometry()
        errs.append(np.sqrt(np.einsum("es,s,es->", g.J, d.ref.sp_w, (U[..., 0] - ex) ** 2)))
    assert errs[1] < 0.05
    assert np.log2(errs[0] / errs[1]) > p + 0.5


def _rate_error(state_fn, exact_fn, n, p, mu=0.01):
    """Max error of the viscous part of the residual, R(mu) - R(0) (the
    inviscid discretisation error cancels), against a closed form."""
    two_pi = 2 * np.pi
    m = M.periodic_box(2, (n, n), (0, 0), (two_pi, two_pi))
    d = FRDiscretisation(m, p, NavierStokes(2, mu=mu, viscous=True))
    d0 = FRDiscretisation(m, p, NavierStokes(2, mu=0.0, viscous=False))
    x = d.sol_coords()
    U = state_fn(x)
    R = d.residual(U) - d0.residual(U)
    ex = exact_fn(x)
    return np.abs(R - ex).max(), R, ex


def test_shear_wave_viscous_residual_closed_form_and_heating():
    mu, U0, k, p0 = 0.01, 0.2, 1.0, 10.0

    def state(x):
        y = x[..., 1]
        rho = np.ones_like(y)
        vel = np.stack([U0 * np.sin(k * y), np.zeros_like(y)], -1)
        return S.primitive_to_conserved(rho, vel, np.full_like(y, p0))

    def exact(x):
        y = x[..., 1]
        out = np.zeros(x.shape[:-1] + (4,))
        out[..., 1] = -mu * U0 * k * k * np.sin(k * y)          # d tau_xy / dy
        out[..., 3] = mu * U0 * U0 * k * k * np.cos(2 * k * y)  # d (u tau_xy) / dy
        return out

    e8, _, _ = _rate_error(state, exact, 8, 4, mu)
    e16, R, ex = _rate_error(state, exact, 16, 4, mu)
    for v in (1, 3):
        err = np.abs(R[..., v] - ex[..., v]).max()
        assert err < 0.05 * np.abs(ex[..., v]).max()
    assert e8 / e16 > 4
    # internal-energy rate d(rho E)/dt - u d(rho u)/dt equals the
    # dissipation mu (du/dy)^2 >= 0 (the printed sign of v_i tau_ij would
    # give a negative rate where the shear is largest)
    x = np.asarray(R.shape)
    m = M.periodic_box(2, (16, 16), (0, 0), (2 * np.pi, 2 * np.pi))
    d = FRDiscretisation(m, 4, NavierStokes(2, mu=mu, viscous=True))
    d0 = FRDiscretisation(m, 4, NavierStokes(2))
    x = d.sol_coords()
    R = d.residual(state(x)) - d0.residual(state(x))
    u = U0 * np.sin(k * x[..., 1])
    heat = R[..., 3] - u * R[..., 1]
    diss = mu * (U0 * k * np.cos(k * x[..., 1])) ** 2
    assert np.abs(heat - diss).max() < 0.05 * diss.max()


def test_resting_temperature_field_conducts_heat_from_hot_to_cold():
    import sympy as sp
    mu, pr, g, p0, eps = 0.05, 0.71, 1.4, 5.0, 0.1
    X = sp.symbols("x")
    rho_expr = 1 + eps * sp.cos(X)
    h_expr = g / (g - 1) * p0 / rho_expr          # E + p/rho - v.v/2 at rest
    rate = sp.lambdify(X, (mu / pr) * sp.diff(h_expr, X, 2), "numpy")

    def state(x):
        xx = x[..., 0]
        rho = 1 + eps * np.cos(xx)
        return S.primitive_to_conserved(rho, np.zeros(xx.shape + (2,)), np.full_like(xx, p0))

    def exact(x):
        out = np.zeros(x.shape[:-1] + (4,))
        out[..., 3] = rate(x[..., 0])
        return out

    e8, _, _ = _rate_error(state, exact, 8, 4, mu)
    e16, R16, ex16 = _rate_error(state, exact, 16, 4, mu)
    assert e16 < 0.02 * np.abs(ex16).max() and e8 / e16 > 4
    # hot where rho is low (x = pi): it must cool there
    m = M.periodic_box(2, (8, 8), (0, 0), (2 * np.pi, 2 * np.pi))
    d = FRDiscretisation(m, 4, NavierStokes(2, mu=mu, viscous=True))
    x = d.sol_coords()
    R = d.residual(state(x))
    hot = np.abs(x[..., 0] - np.pi) < 0.3
    assert np.all(R[..., 3][hot] < 0)


def test_rusanov_consistency_and_skew_symmetry():
    ph = NavierStokes(3)
    rng = np.random.default_rng(3)
    uL = S.random_state(5, 1, 3, 0.4, amp=0.2, seed=1)[:, 0]
    uR = S.random_state(5, 1, 3, 0.4, amp=0.2, seed=2)[:, 0]
    n = rng.normal(size=(5, 3))
    Fc = ph.rusanov(uL, uL, n)
    Fp = np.einsum("ejv,ej->ev", ph.inviscid_flux(uL), n)
    assert np.allclose(Fc, Fp, rtol=1e-15, atol=1e-13)
    assert np.array_equal(ph.rusanov(uL, uR, n), -ph.rusanov(uR, uL, -n))


def test_wall_ghost_gives_zero_mass_and_energy_flux():
    ph = NavierStokes(2)
    uL = S.random_state(7, 1, 2, 0.3, amp=0.3, seed=4)[:, 0]
    n = np.random.default_rng(1).normal(size=(7, 2))
    nhat = n / np.linalg.norm(n, axis=1)[:, None]
    F = ph.rusanov(uL, ph.wall_ghost(uL, nhat), n)
    assert np.abs(F[:, 0]).max() < 1e-13
    assert np.abs(F[:, -1]).max() < 1e-12


@pytest.mark.parametrize("tag", [M.TAG_FARFIELD, M.TAG_INFLOW, M.TAG_OUTFLOW])
def test_farfield_boundaries_keep_the_free_stream(tag):
    m = M.periodic_box(2, (3, 3), (0, 0), (1, 1), jitter=0.2)
    m.face_tag[m.face_tag == M.TAG_PERIODIC] = tag
    mach = 0.2
    ph = NavierStokes(2, mu=0.01, viscous=True, rho_inf=1.0, v_inf=(1.0, 0.0),
                      p_inf=1 / (1.4 * mach ** 2))
    d = FRDiscretisation(m, 3, ph)
    x = d.sol_coords()
    U = S.free_stream(x.shape[:-1], 2, mach)
    assert np.abs(d.residual(U)).max() < 1e-10


def test_uniform_pressure_on_closed_body_gives_zero_force():
    m = M.naca_omesh(0.03, 0.35, 0.1, 4.0, 800, p_geo=3)
    ph = NavierStokes(2, mu=0.001, viscous=True)
    d = FRDiscretisation(m, 3, ph)
    x = d.sol_coords()
    U = S.primitive_to_conserved(np.ones(x.shape[:-1]), np.zeros(x.shape), np.full(x.shape[:-1], 30.0))
    F = d.wall_force(U)
    assert np.abs(F).max() < 1e-11 * 30.0


def test_probe_at_solution_point_and_polynomial_field():
    m = M.periodic_box(2, (3, 2), (0, 0), (3, 2))
    d = FRDiscretisation(m, 3, NavierStokes(2))
    x = d.sol_coords()
    U = S.smooth_perturbed(x, 2, 0.3, amp=0.1)
    pr = Probe(d, x[4, 5])
    assert pr.elem == 4
    assert np.allclose(pr.state(U), U[4, 5], atol=1e-13)
    # degree-3 field in each coordinate is interpolated exactly
    f = lambda X: 1 + 0.1 * X[..., 0] ** 3 - 0.05 * X[..., 0] * X[..., 1] ** 2
    V = np.repeat(f(x)[..., None], 4, axis=-1)
    pt = np.array([1.37, 0.61])
    pr = Probe(d, pt)
    assert np.allclose(pr.state(V), f(pt), atol=1e-13)


def test_characteristic_boundary_state_carries_the_right_invariants():
    """The ghost state keeps the outgoing invariant v_n + 2c/(gamma-1) of the
    interior, takes the incoming invariant v_n - 2c/(gamma-1) of the reference
    state, and the entropy p/rho^gamma and tangential velocity of the upwind
    side."""
    g = 1.4
    ph = NavierStokes(2, rho_inf=1.0, v_inf=(1.0, 0.0), p_inf=1 / (g * 0.3 ** 2))
    rng = np.random.default_rng(11)
    uL = S.random_state(40, 1, 2, 0.3, amp=0.3, seed=3)[:, 0]
    n = rng.normal(size=(40, 2))
    nhat = n / np.linalg.norm(n, axis=1)[:, None]
    vref = np.broadcast_to(ph.v_inf, (40, 2))
    ub = ph.riemann_state(uL, nhat, vref)
    rL, vL, pL = ph.primitives(uL)
    rb, vb, pb = ph.primitives(ub)
    cL, cb = np.sqrt(g * pL / rL), np.sqrt(g * pb / rb)
    c_inf = np.sqrt(g * ph.p_inf / ph.rho_inf)
    vnL, vnb, vnr = (np.sum(v * nhat, 1) for v in (vL, vb, vref))
    assert np.allclose(vnb + 2 * cb / (g - 1), vnL + 2 * cL / (g - 1), rtol=1e-12)
    assert np.allclose(vnb - 2 * cb / (g - 1), vnr - 2 * c_inf / (g - 1), rtol=1e-12, atol=1e-12)
    out = vnb > 0
    s_b = pb / rb ** g
    assert np.allclose(s_b[out], (pL / rL ** g)[out], rtol=1e-12)
    assert np.allclose(s_b[~out], ph.p_inf / ph.rho_inf ** g, rtol=1e-12)
    tb = vb - vnb[:, None] * nhat
    assert np.allclose(tb[out], (vL - vnL[:, None] * nhat)[out], atol=1e-12)
    assert np.allclose(tb[~out], (vref - vnr[:, None] * nhat)[~out], atol=1e-12)


def test_inflow_reference_state_is_the_tanh_profile():
    """At an inflow point of height y the reference velocity is
    U tanh(3 (y - y_wall) / delta) along the free stream: an interior state
    equal to that reference passes through the characteristic construction
    unchanged, and a state with the uniform free stream does not."""
    delta, ywall, mach = 0.2, 0.1, 0.15
    p_inf = 1 / (1.4 * mach ** 2)
    ph = NavierStokes(2, rho_inf=1.0, v_inf=(1.0, 0.0), p_inf=p_inf, inflow_delta=delta,
                      inflow_ywall=ywall)
    y = np.linspace(ywall + 0.01, ywall + 1.0, 25)
    x = np.stack([np.zeros_like(y), y], -1)
    n = np.tile([-0.3, 0.0], (y.size, 1))              # inflow face, outward -x
    prof = np.tanh(3.0 * (y - ywall) / delta)
    uL = S.primitive_to_conserved(np.ones(y.size), np.stack([prof, 0 * y], -1), np.full(y.size, p_inf))
    ghost, ub = ph.boundary_states(M.TAG_INFLOW, uL, n, x)
    assert np.allclose(ghost, uL, rtol=1e-13, atol=1e-13)
    assert np.allclose(ub, uL, rtol=1e-13, atol=1e-13)
    uni = S.primitive_to_conserved(np.ones(y.size), np.stack([np.ones(y.size), 0 * y], -1),
                                   np.full(y.size, p_inf))
    g2, _ = ph.boundary_states(M.TAG_INFLOW, uni, n, x)
    low = prof < 0.9
    assert np.all(np.abs(g2[low, 1] - uni[low, 1]) > 1e-3)


def test_wall_force_linear_shear_is_exact():
    """u = a y over a flat no-slip wall at y = 0: the wall shear stress is
    mu a, so the x-force on a wall of length L is mu a L (p uniform gives no
    net x-force; the linear field is represented exactly for p >= 1)."""
    a, mu, L = 0.7, 0.01, 2.0
    m = M.periodic_box(2, (4, 2), (0.0, 0.0), (L, 1.0))
    m.face_tag = m.face_tag.copy()
    for e in range(m.n_elem):
        xs = m.xyz[m.elem_vert[e]]
        if np.isclose(xs[:, 1].min(), 0.0):
            m.face_tag[e, 2] = M.TAG_WALL
        if np.isclose(xs[:, 1].max(), 1.0):
            m.face_tag[e, 3] = M.TAG_FARFIELD
    ph = NavierStokes(2, mu=mu, viscous=True, rho_inf=1.0, v_inf=(1.0, 0.0), p_inf=10.0)
    d = FRDiscretisation(m, 2, ph)
    x = d.sol_coords()
    U = S.primitive_to_conserved(np.ones(x.shape[:-1]), np.stack([a * x[..., 1], 0 * x[..., 1]], -1),
                                 np.full(x.shape[:-1], 10.0))
    F = d.wall_force(U)
    assert abs(F[0] - mu * a * L) < 1e-12
    # pressure on the wall pushes into it (-y is the fluid's outward normal)
    assert abs(F[1] - (-10.0 * L)) < 1e-11


def test_roe_wave_decomposition_reproduces_the_flux_jump():
    """Roe's property: the signed wave sum sum_k lambda_k alpha_k r_k of the
    Roe-averaged linearisation equals (F(u_R) - F(u_L)) . n_hat exactly."""
    for dim in (2, 3):
        ph = NavierStokes(dim, flux="roe")
        rng = np.random.default_rng(dim)
        uL = S.random_state(30, 1, dim, 0.5, amp=0.4, seed=5)[:, 0]
        uR = S.random_state(30, 1, dim, 0.5, amp=0.4, seed=6)[:, 0]
        n = rng.normal(size=(30, dim))
        nhat = n / np.linalg.norm(n, axis=1)[:, None]
        lam, alpha, R, _ = ph.roe_waves(uL, uR, nhat)
        jump = np.einsum("ek,ek,ekv->ev", lam, alpha, R)
        dF = np.einsum("ejv,ej->ev", ph.inviscid_flux(uR) - ph.inviscid_flux(uL), nhat)
        assert np.allclose(jump, dF, rtol=1e-12, atol=1e-12 * np.abs(dF).max())
        # and the strengths decompose the state jump itself
        du = np.einsum("ek,ekv->ev", alpha, R)
        assert np.allclose(du, uR - uL, rtol=1e-12, atol=1e-12)


def test_roe_consistency_skew_symmetry_and_upwinding():
    ph = NavierStokes(2, flux="roe")
    rng = np.random.default_rng(9)
    uL = S.random_state(20, 1, 2, 0.4, amp=0.2, seed=1)[:, 0]
    uR = S.random_state(20, 1, 2, 0.4, amp=0.2, seed=2)[:, 0]
    n = rng.normal(size=(20, 2))
    assert np.allclose(ph.roe(uL, uL, n), np.einsum("ejv,ej->ev", ph.inviscid_flux(uL), n),
                       rtol=1e-14, atol=1e-12)
    assert np.allclose(ph.roe(uL, uR, n), -ph.roe(uR, uL, -n), rtol=1e-13, atol=1e-12)
    # supersonic flow along +n: the common flux is the upwind (left) flux
    sup = S.primitive_to_conserved(np.ones(3), np.array([[3.0, 0.0]] * 3), np.ones(3))
    sup2 = S.primitive_to_conserved(np.full(3, 1.1), np.array([[3.2, 0.1]] * 3), np.full(3, 1.2))
    nx = np.array([[1.0, 0.0]] * 3)
    assert np.allclose(ph.roe(sup, sup2, nx), np.einsum("ejv,ej->ev", ph.inviscid_flux(sup), nx))


@pytest.mark.parametrize("flux", ["roe"])
def test_roe_scheme_preserves_free_stream_conserves_and_matches_dgsem(flux):
    m = M.vortex_mesh(4, jitter=0.2)
    d = FRDiscretisation(m, 3, NavierStokes(2, mu=0.02, viscous=True, flux=flux))
    assert _fs_max(d) < 1e-11
    g = d.geometry()
    U = S.random_state(m.n_elem, d.ref.nsp, 2, 0.3, amp=0.1)
    R = d.residual(U)
    tot = np.einsum("es,s,esv->v", g.J, d.ref.sp_w, R)
    scale = np.einsum("es,s,esv->v", g.J, d.ref.sp_w, np.abs(R))
    assert np.all(np.abs(tot) < 1e-13 * scale)


@pytest.mark.slow
def test_roe_vortex_converges_at_design_order():
    def err(n):
        m = M.vortex_mesh(n)
        d = FRDiscretisation(m, 3, NavierStokes(2, flux="roe"))
        x = d.sol_coords()
        U = S.isentropic_vortex(x)
        for _ in range(20):
            U = T.rk4_step(d.residual, U, 5e-3)
        ex = S.isentropic_vortex(x, t=0.1)
        g = d.geometry()
        return np.sqrt(np.einsum("es,s,es->", g.J, d.ref.sp_w, (U - ex)[..., 0] ** 2))
    assert np.log2(err(16) / err(32)) > 3.6


def test_ldg_conserves_preserves_free_stream_and_has_single_valued_common_solution():
    m = M.vortex_mesh(4, jitter=0.2)
    d = FRDiscretisation(m, 3, NavierStokes(2, mu=0.03, viscous=True), viscous_scheme="ldg")
    assert _fs_max(d) < 1e-11
    g = d.geometry()
    U = S.random_state(m.n_elem, d.ref.nsp, 2, 0.3, amp=0.1)
    R = d.residual(U)
    tot = np.einsum("es,s,esv->v", g.J, d.ref.sp_w, R)
    scale = np.einsum("es,s,esv->v", g.J, d.ref.sp_w, np.abs(R))
    assert np.all(np.abs(tot) < 1e-13 * scale)
    # every interface has exactly one left side
    own = np.arange(m.n_elem)[:, None] * d.ref.nfp + np.arange(d.ref.nfp)[None, :]
    pe, pf = d.partner // d.ref.nfp, d.partner % d.ref.nfp
    assert np.all(d.side + d.side[pe, pf] == 0)
    assert np.all((d.side > 0) == (own < d.partner))


@pytest.mark.slow
@pytest.mark.parametrize("p", [2, 3])
def test_ldg_heat_equation_decay_converges(p):
    nu, t_end, steps = 0.1, 1.0, 400
    errs = []
    for n in (4, 8):
        m = M.periodic_box(2, (n, n), (0, 0), (2 * np.pi, 2 * np.pi))
        d = FRDiscretisation(m, p, ScalarDiffusion(2, nu), viscous_scheme="ldg")
        x = d.sol_coords()
        U = (np.sin(x[..., 0]) * np.sin(x[..., 1]))[..., None]
        for _ in range(steps):
            U = T.rk4_step(d.residual, U, t_end / steps)
        ex = np.exp(-2 * nu * t_end) * np.sin(x[..., 0]) * np.sin(x[..., 1])
        g = d.geometry()
        errs.append(np.sqrt(np.einsum("es,s,es->", g.J, d.ref.sp_w, (U[..., 0] - ex) ** 2)))
    assert errs[1] < 0.05
    assert np.log2(errs[0] / errs[1]) > p + 0.5
