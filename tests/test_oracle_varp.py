"""Pins of the variable-degree oracle (``oracle.fr_var``) against facts that
do not come from it: the uniform-degree oracle (itself pinned), polynomial
exactness of the mortar operators in every relative face orientation,
free-stream preservation, discrete conservation, a single-valued LDG common
solution across mortars, and the convergence rate of the residual on the
isentropic vortex."""
import numpy as np
import pytest

from synth import meshes as M, states as S
from oracle.fr import FRDiscretisation
from oracle.fr_var import VarFRDiscretisation
from oracle.physics import NavierStokes


def _phys(dim, viscous, mach=0.3, flux="rusanov", mu=0.01):
    return NavierStokes(dim, gamma=1.4, mu=mu if viscous else 0.0, prandtl=0.71, viscous=viscous,
                        rho_inf=1.0, v_inf=(1.0, 0.0, 0.0)[:dim], p_inf=1.0 / (1.4 * mach ** 2),
                        flux=flux)


DEGREE_SETS = [(1, 2, 3, 4), (0, 1, 2, 3)]


def _mixed_box(dim, jitter, seed=5, degrees=(1, 2, 3, 4)):
    n = (6, 5) if dim == 2 else (3, 3, 2)
    m = M.reorient(M.periodic_box(dim, n, (0.0,) * dim, (1.0,) * dim, jitter=jitter), seed)
    return m, M.checker_degrees(m, degrees, seed=seed)


@pytest.mark.parametrize("scheme,flux", [("br2", "rusanov"), ("ldg", "rusanov"), ("br2", "roe")])
def test_uniform_degree_is_the_fr_oracle(scheme, flux):
    m = M.cavity_mesh(300)
    ph = _phys(2, True, flux=flux)
    d0 = FRDiscretisation(m, 3, ph, viscous_scheme=scheme)
    d1 = VarFRDiscretisation(m, np.full(m.n_elem, 3), ph, viscous_scheme=scheme)
    u = S.smooth_perturbed(d0.sol_coords(), 2, 0.3, amp=0.05, seed=1)
    R0 = d0.residual(u)
    R1 = d1.residual(u.reshape(-1, 4)).reshape(R0.shape)
    assert np.linalg.norm(R1 - R0) <= 1e-14 * np.linalg.norm(R0)
    assert np.allclose(d1.wall_force(u.reshape(-1, 4)), d0.wall_force(u), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("degrees", DEGREE_SETS)
@pytest.mark.parametrize("dim", [2, 3])
def test_mortar_operators_are_exact_on_polynomials_in_every_orientation(dim, degrees):
    """T carries a degree-p_lo polynomial of the physical coordinates from the
    lower side's points to the higher side's; P carries it back unchanged
    and keeps the face integral of any trace (affine faces, all relative
    orientations from randomly rotated element frames)."""
    m, ep = _mixed_box(dim, jitter=0.0, degrees=degrees)
    d = VarFRDiscretisation(m, ep, _phys(dim, False))
    rng = np.random.default_rng(0)
    seen = {"hi": 0, "lo": 0}
    for (e, fc), (kind, e2, fc2, X) in d.links.items():
        if kind == "same" or m.face_tag[e, fc] == 1:
            continue
        q, q2 = int(ep[e]), int(ep[e2])
        r, r2 = d.refq[q], d.refq[q2]
        x_own = d.geo[q].x_fp[d.loc[e], fc * r.nfpf:(fc + 1) * r.nfpf]
        x_oth = d.geo[q2].x_fp[d.loc[e2], fc2 * r2.nfpf:(fc2 + 1) * r2.nfpf]
        deg = min(q, q2)
        c = rng.standard_normal((deg + 1,) * dim)

        def f(x):
            out = np.zeros(len(x))
            for idx in np.ndindex(*c.shape):
                if sum(idx) <= deg:
                    out += c[idx] * np.prod([x[:, a] ** idx[a] for a in range(dim)], axis=0)
            return out

        assert np.max(np.abs(X @ f(x_oth) - f(x_own))) < 1e-11 * np.max(np.abs(f(x_own)))
        if kind == "lo":
            g = rng.standard_normal(r2.nfpf)
            w_own = r.fp_w[fc * r.nfpf:(fc + 1) * r.nfpf]
            w_oth = r2.fp_w[fc2 * r2.nfpf:(fc2 + 1) * r2.nfpf]
            assert abs(w_own @ (X @ g) - w_oth @ g) < 1e-13 * np.abs(w_oth @ np.abs(g))
        seen[kind] += 1
    assert seen["hi"] > 10 and seen["lo"] > 10


@pytest.mark.parametrize("degrees", DEGREE_SETS)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("viscous,scheme", [(False, "br2"), (True, "br2"), (True, "ldg")])
def test_free_stream_preserved_on_mixed_degrees(dim, viscous, scheme, degrees):
    m, ep = _mixed_box(dim, jitter=0.2, degrees=degrees)
    d = VarFRDiscretisation(m, ep, _phys(dim, viscous), viscous_scheme=scheme)
    u = S.free_stream((d.n_sp,), dim, 0.3, direction=(1.0, 0.4, 0.2)[:dim])
    R, mag = d.residual(u, magnitude=True)
    assert np.max(np.abs(R)) < 1e-13 * np.max(mag)


@pytest.mark.parametrize("degrees", DEGREE_SETS)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("scheme,flux", [("br2", "rusanov"), ("ldg", "rusanov"), ("br2", "roe")])
def test_mixed_degree_meshes_conserve(dim, scheme, flux, degrees):
    m, ep = _mixed_box(dim, jitter=0.2, degrees=degrees)
    d = VarFRDiscretisation(m, ep, _phys(dim, True, flux=flux), viscous_scheme=scheme)
    u = S.smooth_perturbed(d.sol_coords(), dim, 0.3, amp=0.05, seed=2)
    R = d.residual(u)
    assert np.all(np.abs(d.integral(R)) < 1e-13 * d.integral(np.abs(R)).max())


def test_ldg_common_solution_is_single_valued_across_mortars():
    """On the lower side the common solution equals the projection of the
    higher side's: the one-sided switch agrees on both sides."""
    m, ep = _mixed_box(2, jitter=0.2)
    d = VarFRDiscretisation(m, ep, _phys(2, True), viscous_scheme="ldg", ldg_beta=0.5)
    u = S.smooth_perturbed(d.sol_coords(), 2, 0.3, amp=0.05, seed=4)
    Ub = d.blocks(u)
    Uf = {q: np.einsum("fs,esv->efv", d.refq[q].M0, Ub[q]) for q in d.degrees}
    uR, _ = d._partner_traces(Uf)
    uc = {q: (0.5 + 0.5 * d.side[q])[..., None] * Uf[q] + (0.5 - 0.5 * d.side[q])[..., None] * uR[q]
          for q in d.degrees}
    n = 0
    for (e, fc), (kind, e2, fc2, X) in d.links.items():
        if kind != "lo":
            continue
        q, q2 = int(ep[e]), int(ep[e2])
        r, r2 = d.refq[q], d.refq[q2]
        lo = uc[q][d.loc[e], fc * r.nfpf:(fc + 1) * r.nfpf]
        hi = uc[q2][d.loc[e2], fc2 * r2.nfpf:(fc2 + 1) * r2.nfpf]
        assert np.allclose(lo, X @ hi, rtol=1e-13, atol=1e-13)
        n += 1
    assert n > 10


def _vortex_residual_error(n, degrees):
    m = M.vortex_mesh(n)
    d = VarFRDiscretisation(m, M.checker_degrees(m, degrees, seed=7),
                            NavierStokes(2, gamma=1.4, v_inf=(1.0, 0.0), p_inf=1.0))
    x = d.sol_coords()
    h = 1e-5
    dudt = (S.isentropic_vortex(x, t=h) - S.isentropic_vortex(x, t=-h)) / (2 * h)
    return float(np.sqrt(d.integral((d.residual(S.isentropic_vortex(x)) - dudt) ** 2).sum()))


@pytest.mark.parametrize("p", [2, 3])
def test_mixed_degree_vortex_residual_converges_like_its_lower_degree(p):
    """Residual error against the exact du/dt of the advected vortex: a
    random mix of degrees p and p+1 converges at the order of degree p and is
    no worse than degree p everywhere (a mis-oriented or inconsistent mortar
    leaves an O(1) error that does not converge)."""
    e16, e32 = _vortex_residual_error(16, (p, p + 1)), _vortex_residual_error(32, (p, p + 1))
    u32 = _vortex_residual_error(32, (p,))
    assert np.log2(e16 / e32) > p - 0.3
    assert e32 < 1.05 * u32


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_degree_zero_is_first_order_finite_volume(flux):
    """With one solution point per element and the DG-recovery correction
    (g_L' = -1/2, g_R' = 1/2), FR reduces to the cell-centred first-order
    finite-volume scheme: on straight-edged (bilinear) quads
    du/dt = -(1/area) sum over edges of F*(u, u_neighbour, n) |edge|.  The
    right-hand side is written out here from the vertex coordinates."""
    from oracle.geometry import face_pairs
    m = M.periodic_box(2, (7, 6), (0.0, 0.0), (1.4, 1.0), jitter=0.25)
    ph = _phys(2, False, flux=flux)
    d = VarFRDiscretisation(m, np.zeros(m.n_elem, dtype=np.int64), ph)
    u = S.smooth_perturbed(d.sol_coords(), 2, 0.3, amp=0.1, seed=6)
    X = m.xyz[m.elem_vert]                                   # corners, tensor order
    ring = [0, 1, 3, 2]                                      # counter-clockwise
    P = X[:, ring]
    area = 0.5 * np.sum(P[:, :, 0] * np.roll(P[:, :, 1], -1, 1) - np.roll(P[:, :, 0], -1, 1) * P[:, :, 1], 1)
    edge = {0: (2, 0), 1: (1, 3), 2: (0, 1), 3: (3, 2)}      # face -> corners, counter-clockwise
    nb = {(e, f): e2 for (e, f, e2, f2, sh) in face_pairs(m)}
    R = np.zeros_like(u)
    for e in range(m.n_elem):
        for f, (a, b) in edge.items():
            t = X[e, b] - X[e, a]
            n = np.array([t[1], -t[0]])                      # outward, |n| = edge length
            R[e] -= ph.common_inviscid(u[e][None], u[nb[(e, f)]][None], n[None])[0]
        R[e] /= area[e]
    assert np.abs(d.residual(u) - R).max() < 1e-12 * np.abs(R).max()
