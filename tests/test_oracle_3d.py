"""Pins of the oracle's three-dimensional viscous terms (Sec. 2.1, Eqs. 1-7)
and of its metric terms on curved, spanwise-extruded hexahedra (the FR
geometry of Sec. 2.3), against closed forms of the continuous equations:

* a shear wave v_a = U sin(k x_b) for every ordered pair of directions
  (a, b), a != b: the viscous part of the residual is d tau_ab / d x_b in
  momentum a and d (v_a tau_ab) / d x_b in energy;
* a longitudinal wave v_a = U sin(k x_a) in every direction: it fixes the
  dilatation term of tau (tau_aa = 4/3 mu dv_a/dx_a);
* a resting density (temperature) field along z: the energy rate is the
  printed heat-flux divergence (mu/Pr) d^2/dz^2 (E + p/rho);
* the Taylor-Green vortex at t = 0: the exact kinetic-energy rate of a
  divergence-free periodic field is -mu int |omega|^2 = -(3/4) mu (2 pi)^3;
* free stream on tandem-cylinder meshes (curved O-rings, degree-2 geometry,
  extruded along the span) for every p >= 1, and on hexes curved in all
  three directions exactly when p >= 2q - 2 (Gauss quadrature of the
  constant-flux identity exact), disturbed below that.

A planted mistake (a wrong third-component index in the stress tensor) fails
these pins.
"""
import numpy as np
import pytest

from synth import meshes as M, states as S
from oracle.fr import FRDiscretisation
from oracle.physics import NavierStokes

TWO_PI = 2 * np.pi
_DIR = np.array([1.0, 0.3, 0.2]) / np.linalg.norm([1.0, 0.3, 0.2])


def _viscous_part(phys_cls, n, b, p, state_fn, mu):
    """R(mu) - R(0) on a periodic (2 pi)^3 box with n elements along
    direction b and one across the others (the fields below vary along b
    only): the viscous part of the residual, the inviscid discretisation
    error cancelling."""
    counts = [1, 1, 1]
    counts[b] = n
    m = M.periodic_box(3, tuple(counts), (0, 0, 0), (TWO_PI, TWO_PI, TWO_PI))
    d = FRDiscretisation(m, p, phys_cls(3, mu=mu, viscous=True))
    d0 = FRDiscretisation(m, p, phys_cls(3, mu=0.0, viscous=False))
    x = d.sol_coords()
    U = state_fn(x)
    return x, d.residual(U) - d0.residual(U), d


def _shear_state(a, b, U0, k, p0):
    def state(x):
        rho = np.ones(x.shape[:-1])
        vel = np.zeros(x.shape)
        vel[..., a] = U0 * np.sin(k * x[..., b])
        return S.primitive_to_conserved(rho, vel, np.full_like(rho, p0))
    return state


def _shear_errors(phys_cls, n=24, p=4, mu=0.01, U0=0.2, k=1.0, p0=10.0):
    """Worst error of the shear-wave closed form over all six ordered
    direction pairs, relative to each component's amplitude: momentum a
    (mu U k^2) and energy (mu U^2 k^2)."""
    worst = 0.0
    for a in range(3):
        for b in range(3):
            if a == b:
                continue
            x, R, _ = _viscous_part(phys_cls, n, b, p, _shear_state(a, b, U0, k, p0), mu)
            xb = x[..., b]
            ex = np.zeros(R.shape)
            ex[..., 1 + a] = -mu * U0 * k * k * np.sin(k * xb)
            ex[..., 4] = mu * U0 * U0 * k * k * np.cos(2 * k * xb)
            scale = np.full(5, mu * U0 * k * k)
            scale[4] = mu * U0 * U0 * k * k
            worst = max(worst, float((np.abs(R - ex) / scale).max()))
    return worst


def _longitudinal_errors(phys_cls, n=24, p=4, mu=0.01, U0=0.1, k=1.0, p0=10.0):
    worst = 0.0
    for a in range(3):
        def state(x, a=a):
            rho = np.ones(x.shape[:-1])
            vel = np.zeros(x.shape)
            vel[..., a] = U0 * np.sin(k * x[..., a])
            return S.primitive_to_conserved(rho, vel, np.full_like(rho, p0))
        x, R, _ = _viscous_part(phys_cls, n, a, p, state, mu)
        xa = x[..., a]
        ex = np.zeros(R.shape)
        # tau_aa = 4/3 mu U k cos(k x_a); the other normal stresses depend on
        # x_a only and are differentiated along their own direction (zero)
        ex[..., 1 + a] = -(4.0 / 3.0) * mu * U0 * k * k * np.sin(k * xa)
        ex[..., 4] = (4.0 / 3.0) * mu * U0 * U0 * k * k * np.cos(2 * k * xa)
        scale = np.full(5, (4.0 / 3.0) * mu * U0 * k * k)
        scale[4] = (4.0 / 3.0) * mu * U0 * U0 * k * k
        worst = max(worst, float((np.abs(R - ex) / scale).max()))
    return worst


def test_3d_shear_waves_in_every_orientation_match_the_closed_form():
    e = _shear_errors(NavierStokes)
    assert e < 0.03, e


def test_3d_shear_wave_viscous_residual_converges():
    errs = []
    for n in (8, 16):
        x, R, _ = _viscous_part(NavierStokes, n, 0, 3, _shear_state(2, 0, 0.2, 1.0, 10.0), 0.01)
        ex = np.zeros(R.shape)
        ex[..., 3] = -0.01 * 0.2 * np.sin(x[..., 0])
        ex[..., 4] = 0.01 * 0.04 * np.cos(2 * x[..., 0])
        errs.append(np.abs(R - ex).max())
    assert errs[1] < errs[0] / 4, errs


def test_3d_longitudinal_waves_fix_the_dilatation_term():
    e = _longitudinal_errors(NavierStokes)
    assert e < 0.03, e


def test_3d_resting_temperature_field_along_z_conducts_heat():
    import sympy as sp
    mu, pr, g, p0, eps = 0.05, 0.71, 1.4, 5.0, 0.1
    Z = sp.symbols("z")
    h_expr = g / (g - 1) * p0 / (1 + eps * sp.cos(Z))      # E + p/rho - v.v/2 at rest
    rate = sp.lambdify(Z, (mu / pr) * sp.diff(h_expr, Z, 2), "numpy")

    def state(x):
        rho = 1 + eps * np.cos(x[..., 2])
        return S.primitive_to_conserved(rho, np.zeros(x.shape), np.full_like(rho, p0))

    x, R, _ = _viscous_part(NavierStokes, 16, 2, 4, state, mu)
    ex = rate(x[..., 2])
    assert np.abs(R[..., :4]).max() < 1e-12
    assert np.abs(R[..., 4] - ex).max() < 0.03 * np.abs(ex).max()
    # hottest (lowest density) plane z = pi must cool
    hot = np.abs(x[..., 2] - np.pi) < 0.3
    assert np.all(R[..., 4][hot] < 0)


def _tgv_rates(n, p=3, mu=1.0 / 1600.0, mach=0.1):
    """Discrete kinetic-energy rate of the Taylor-Green field at t = 0 from
    the full residual and from its viscous part alone."""
    m = M.tgv_mesh(n)
    p_inf = 1.0 / (1.4 * mach * mach)
    ph = NavierStokes(3, mu=mu, viscous=True, p_inf=p_inf)
    d = FRDiscretisation(m, p, ph)
    d0 = FRDiscretisation(m, p, NavierStokes(3, mu=0.0, viscous=False, p_inf=p_inf))
    x = d.sol_coords()
    U = S.taylor_green(x, mach=mach)
    R = d.residual(U)
    Rv = R - d0.residual(U)
    g = d.geometry()
    rho = U[..., 0]
    v = U[..., 1:4] / rho[..., None]

    def rate(Rx):
        dek = np.einsum("esi,esi->es", v, Rx[..., 1:4]) - 0.5 * np.sum(v * v, -1) * Rx[..., 0]
        return float(np.einsum("es,s,es->", g.J, d.ref.sp_w, dek))
    return rate(R), rate(Rv)


def test_taylor_green_kinetic_energy_rate_converges_to_minus_mu_enstrophy():
    mu = 1.0 / 1600.0
    exact = -0.75 * mu * TWO_PI ** 3
    full6, visc6 = _tgv_rates(6, mu=mu)
    full8, visc8 = _tgv_rates(8, mu=mu)
    ev6, ev8 = abs(visc6 / exact - 1), abs(visc8 / exact - 1)
    ef6, ef8 = abs(full6 / exact - 1), abs(full8 / exact - 1)
    assert ev8 < 2e-5 and ev8 < ev6 / 4, (ev6, ev8)
    assert ef8 < 1e-3 and ef8 < ef6 / 4, (ef6, ef8)


def _free_stream_error(m, p, keep=None):
    ph = NavierStokes(3, mu=1e-3, viscous=True, rho_inf=1.0, v_inf=_DIR,
                      p_inf=1.0 / (1.4 * 0.2 ** 2))
    d = FRDiscretisation(m, p, ph)
    x = d.sol_coords()
    U = S.free_stream(x.shape[:-1], 3, 0.2, direction=_DIR)
    R = d.residual(U)
    if keep is not None:
        R = R[keep(d)]
    return np.abs(R).max() / np.abs(ph.inviscid_flux(U)).max()


def _away_from_walls(d):
    wall = np.any(d.bc == 2, axis=1)
    pe = d.partner_elem[wall].ravel()
    near = np.unique(np.concatenate([np.nonzero(wall)[0], pe[pe >= 0]]))
    keep = np.setdiff1d(np.arange(d.mesh.n_elem), near)
    assert keep.size > d.mesh.n_elem // 2
    return keep


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_free_stream_preserved_on_curved_extruded_tandem_hexes(p):
    """Degree-2 O-rings extruded along the span.  The FR residual of a
    constant flux is a Gauss-quadrature form of int grad(phi).S - int phi n
    (the DG-recovery correction); an extruded map keeps the metric rows of
    degree <= q in each direction, so quadrature is exact, and uniform flow
    preserved, whenever q <= p + 2 (elements touching a cylinder are left
    out: uniform flow does not satisfy no slip)."""
    m = M.tandem_cylinders(3.0, 0.8, 600, n_span=2, q=2)
    assert _free_stream_error(m, p, _away_from_walls) < 1e-11


@pytest.mark.parametrize("q,p,exact", [(2, 1, False), (2, 2, True), (2, 3, True),
                                       (3, 3, False), (3, 4, True)])
def test_free_stream_on_fully_curved_hexes_holds_exactly_when_p_is_at_least_2q_minus_2(q, p, exact):
    """Cross-product metrics of a map curved in all three directions are
    polynomials of degree 2q in their own direction and 2q - 1 across, so
    the quadrature of the constant-flux identity is exact, and the free
    stream preserved to round-off, exactly when p >= 2q - 2; below that it
    is disturbed at the truncation level."""
    err = _free_stream_error(M.curved_periodic_box(3, q), p)
    if exact:
        assert err < 1e-12
    else:
        assert err > 1e-5


class _WrongIndex(NavierStokes):
    """A planted mistake: the z-derivatives read from the y row of the
    gradient (a wrong third-component index)."""

    def viscous_flux(self, u, grad):
        if self.dim == 3:
            g = grad.copy()
            g[..., 2, :] = grad[..., 1, :]
            return super().viscous_flux(u, g)
        return super().viscous_flux(u, grad)


def test_planted_wrong_stress_index_fails_the_3d_pins():
    assert _shear_errors(_WrongIndex) > 0.5
