"""Pins of the oracle's reference element against closed forms and library
routines (Sec. 2.3: Huynh's FR with DG-recovery correction on Gauss-Legendre
points)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import basis
from oracle.element import RefElement


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_legendre_nodes_match_library_and_integrate_exactly(n):
    x, w = basis.gauss_legendre(n)
    xl, wl = npleg.leggauss(n)
    assert np.allclose(x, xl, atol=1e-15, rtol=0)
    assert np.allclose(w, wl, atol=1e-15, rtol=0)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * n):                 # exact for degree <= 2n-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # not exact one degree higher
    k = 2 * n
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_lagrange_interpolation_and_derivative_exact_on_degree_p(p):
    rng = np.random.default_rng(p)
    x, _ = basis.gauss_legendre(p + 1)
    c = rng.normal(size=p + 1)
    f = np.polynomial.Polynomial(c)
    t = np.linspace(-1.3, 1.2, 17)
    L = basis.lagrange(x, t)
    assert np.allclose(L @ f(x), f(t), atol=1e-13)
    dL = basis.lagrange_deriv(x, t)
    assert np.allclose(dL @ f(x), f.deriv()(t), atol=1e-12)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_dg_correction_endpoints_and_dg_identity(p):
    gL, gR, _, _ = basis.correction_dg(p, np.array([-1.0, 1.0]))
    assert np.allclose(gL, [1.0, 0.0], atol=1e-15)
    assert np.allclose(gR, [0.0, 1.0], atol=1e-15)
    # DG identity: g_R'(x_i) = l_i(1)/w_i, g_L'(x_i) = -l_i(-1)/w_i
    x, w = basis.gauss_legendre(p + 1)
    _, _, dgL, dgR = basis.correction_dg(p, x)
    ends = basis.lagrange(x, np.array([-1.0, 1.0]))
    assert np.allclose(dgR, ends[1] / w, atol=1e-12)
    assert np.allclose(dgL, -ends[0] / w, atol=1e-12)
    # right Radau polynomial: g_L vanishes at the p+1 right-Radau points,
    # i.e. it is orthogonal to all polynomials of degree p-1
    xs, ws = basis.gauss_legendre(p + 3)
    gLq, _, _, _ = basis.correction_dg(p, xs)
    for k in range(p):
        assert abs(np.dot(ws, gLq * xs ** k)) < 1e-13


@pytest.mark.parametrize("dim,p", [(2, 0), (2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3), (3, 4)])
def test_element_operators_exact_on_tensor_polynomials(dim, p):
    ref = RefElement(dim, p)
    rng = np.random.default_rng(10 * dim + p)
    # random tensor polynomial of degree p in each variable
    C = rng.normal(size=(p + 1,) * dim)

    def f(X):
        out = np.zeros(X.shape[0])
        for idx in np.ndindex(*C.shape):
            term = C[idx] * np.ones(X.shape[0])
            for a in range(dim):
                term = term * X[:, a] ** idx[a]
            out += term
        return out

    def df(X, k):
        out = np.zeros(X.shape[0])
        for idx in np.ndindex(*C.shape):
            if idx[k] == 0:
                continue
            term = C[idx] * idx[k] * np.ones(X.shape[0])
            for a in range(dim):
                term = term * X[:, a] ** (idx[a] - (1 if a == k else 0))
            out += term
        return out

    u = f(ref.sp_xi)
    assert np.allclose(ref.M0 @ u, f(ref.fp_xi), atol=1e-12)
    for k in range(dim):
        assert np.allclose(ref.D[k] @ u, df(ref.sp_xi, k), atol=1e-11)
    pts = rng.uniform(-1, 1, size=(7, dim))
    assert np.allclose(ref.interp_matrix(pts) @ u, f(pts), atol=1e-12)
    # quadrature weights: face weights integrate 1 over each face
    for face in range(2 * dim):
        sl = slice(face * ref.nfpf, (face + 1) * ref.nfpf)
        assert abs(ref.fp_w[sl].sum() - 2.0 ** (dim - 1)) < 1e-13
    assert abs(ref.sp_w.sum() - 2.0 ** dim) < 1e-13
    # every flux point lies at the end of its line of solution points
    for fidx in range(ref.nfp):
        line = ref.fp_line_sp[fidx]
        k = ref.fp_dir[fidx]
        others = [a for a in range(dim) if a != k]
        assert np.allclose(ref.sp_xi[line][:, others], ref.fp_xi[fidx, others])
