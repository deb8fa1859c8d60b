"""Element maps, metric terms and face connectivity, FP64 (test
infrastructure only).

Reading of the paper's silent points (the paper defers the FR discretisation
to its earlier work, Sec. 2.3):

* the element map x(xi) is the tensor Lagrange interpolant of the geometry
  nodes on the equispaced lattice of degree q (q = 1: the corners);
* metric terms are the adjugate of the map Jacobian A[j, k] = dx_j/dxi_k,
  S[k, j] = J dxi_k/dx_j, evaluated analytically at every point; in 2-D
  S = [[y_eta, -x_eta], [-y_xi, x_xi]], in 3-D row k is the cross product
  dx/dxi_{k+1} x dx/dxi_{k+2} (cyclic);
* the outward normal at a flux point, scaled by the surface Jacobian, is
  n = sign * S[k, :] at that point (k the face direction, sign -1 on a
  - face);
* flux points of two connected faces are paired by physical position (after
  the periodic shift for periodic faces).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import basis

_QUAD_FACES = [(0, 2), (1, 3), (0, 1), (2, 3)]
_HEX_FACES = [(0, 2, 4, 6), (1, 3, 5, 7), (0, 1, 4, 5), (2, 3, 6, 7),
              (0, 1, 2, 3), (4, 5, 6, 7)]


def _shape(q: int, dim: int, X):
    """Tensor equispaced Lagrange shape functions N (npts, nn) and their
    reference derivatives dN (npts, nn, dim) at points X (npts, dim)."""
    eq = np.linspace(-1.0, 1.0, q + 1)
    X = np.atleast_2d(X)
    npts = X.shape[0]
    L = [basis.lagrange(eq, X[:, a]) for a in range(dim)]
    dL = [basis.lagrange_deriv(eq, X[:, a]) for a in range(dim)]
    idx = np.array([t[::-1] for t in itertools.product(range(q + 1), repeat=dim)])
    nn = idx.shape[0]
    N = np.ones((npts, nn))
    dN = np.ones((npts, nn, dim))
    for a in range(dim):
        N *= L[a][:, idx[:, a]]
        for k in range(dim):
            dN[:, :, k] *= (dL[a] if a == k else L[a])[:, idx[:, a]]
    return N, dN


def map_points(mesh, elems, X):
    """Physical coordinates (ne, npts, dim) of reference points X in elems.

    The map is translation invariant (the shape functions sum to one), so it
    is evaluated on node offsets from the element's first node and the
    offset added back: the same value with rounding relative to the element
    size instead of the coordinates' magnitude."""
    nodes = mesh.node_coords()[elems]
    base = nodes[:, :1, :]
    N, _ = _shape(mesh.geo_order, mesh.dim, X)
    return base + np.einsum("pa,eaj->epj", N, nodes - base)


def jacobian(mesh, elems, X):
    """A[e, p, j, k] = dx_j / dxi_k at reference points X (from node offsets:
    the derivative of a translation is zero)."""
    nodes = mesh.node_coords()[elems]
    _, dN = _shape(mesh.geo_order, mesh.dim, X)
    return np.einsum("pak,eaj->epjk", dN, nodes - nodes[:, :1, :])


def adjugate(A):
    """Metric terms S[..., k, j] = J dxi_k/dx_j and J = det A."""
    dim = A.shape[-1]
    S = np.empty_like(A)
    if dim == 2:
        S[..., 0, 0] = A[..., 1, 1]
        S[..., 0, 1] = -A[..., 0, 1]
        S[..., 1, 0] = -A[..., 1, 0]
        S[..., 1, 1] = A[..., 0, 0]
        J = A[..., 0, 0] * A[..., 1, 1] - A[..., 0, 1] * A[..., 1, 0]
    else:
        for k in range(3):
            a = A[..., :, (k + 1) % 3]
            b = A[..., :, (k + 2) % 3]
            S[..., k, :] = np.cross(a, b)
        J = np.einsum("...j,...j->...", A[..., :, 0], S[..., 0, :])
    return S, J


class Geometry:
    """Per-element geometric data for a subset of elements."""

    def __init__(self, mesh, ref, elems):
        elems = np.asarray(elems, dtype=np.int64)
        self.elems = elems
        A = jacobian(mesh, elems, ref.sp_xi)
        self.S, self.J = adjugate(A)                      # (ne,nsp,d,d), (ne,nsp)
        if np.any(self.J <= 0.0):
            raise ValueError("non-positive Jacobian")
        Af = jacobian(mesh, elems, ref.fp_xi)
        Sf, _ = adjugate(Af)
        k = ref.fp_dir
        self.n = Sf[:, np.arange(ref.nfp), k, :] * ref.fp_sign[None, :, None]
        self.x_sp = map_points(mesh, elems, ref.sp_xi)
        self.x_fp = map_points(mesh, elems, ref.fp_xi)


def _face_key_ids(ev, loc):
    return tuple(sorted(int(ev[c]) for c in loc))


def face_pairs(mesh):
    """Every connected face seen from both sides: a list of (e, face, e2,
    face2, shift) with the corners of (e, face) + shift on those of (e2,
    face2).  Interior faces share their corner vertices; periodic faces are
    matched by corner coordinates after adding or subtracting one of the
    mesh's periodic shifts."""
    dim = mesh.dim
    faces = _QUAD_FACES if dim == 2 else _HEX_FACES
    E = mesh.n_elem
    ev = mesh.elem_vert
    tags = mesh.face_tag

    pairs = []          # (e, face, e2, face2, shift vector)
    by_ids = {}
    for e in range(E):
        for fc, loc in enumerate(faces):
            if tags[e, fc] == 0:
                by_ids.setdefault(_face_key_ids(ev[e], loc), []).append((e, fc))
    for key, lst in by_ids.items():
        if len(lst) != 2:
            raise ValueError("interior face without exactly one partner")
        (a, fa), (b, fb) = lst
        pairs.append((a, fa, b, fb, np.zeros(dim)))
        pairs.append((b, fb, a, fa, np.zeros(dim)))

    # periodic faces: match corner sets after a +/- shift
    if np.any(tags == 1):
        span = np.ptp(mesh.xyz, axis=0).max()
        scale = 1e6 / max(span, 1e-300)

        def ckey(pts):
            r = np.round(pts * scale).astype(np.int64)
            return tuple(sorted(map(tuple, r)))

        table = {}
        per = [(e, fc) for e in range(E) for fc in range(2 * dim) if tags[e, fc] == 1]
        for e, fc in per:
            table[ckey(mesh.xyz[ev[e, list(faces[fc])]])] = (e, fc)
        for e, fc in per:
            pts = mesh.xyz[ev[e, list(faces[fc])]]
            found = None
            for s in mesh.periodic_shift:
                for sg in (1.0, -1.0):
                    hit = table.get(ckey(pts + sg * s))
                    if hit is not None and hit != (e, fc):
                        found = (hit, sg * s)
                        break
                if found:
                    break
            if found is None:
                raise ValueError("periodic face without partner")
            (b, fb), sh = found
            pairs.append((e, fc, b, fb, sh))
    return pairs


def connectivity(mesh, ref, tol=1e-8):
    """Partner of every flux point.

    Returns (partner, bc): partner[e, f] = e2 * nfp + f2 for connected flux
    points, or -1 for boundary points; bc[e, f] = face tag (2..5) at boundary
    points, 0 elsewhere."""
    dim = mesh.dim
    E = mesh.n_elem
    nfp, nfpf = ref.nfp, ref.nfpf
    partner = np.full((E, nfp), -1, dtype=np.int64)
    bc = np.zeros((E, nfp), dtype=np.int32)
    tags = mesh.face_tag
    pairs = face_pairs(mesh)

    if pairs:
        pe = np.array([p[0] for p in pairs])
        pf = np.array([p[1] for p in pairs])
        qe = np.array([p[2] for p in pairs])
        qf = np.array([p[3] for p in pairs])
        sh = np.array([p[4] for p in pairs])
        chunk = 20000
        for c0 in range(0, len(pairs), chunk):
            sl = slice(c0, c0 + chunk)
            xa = _face_points(mesh, ref, pe[sl], pf[sl]) + sh[sl, None, :]
            xb = _face_points(mesh, ref, qe[sl], qf[sl])
            d = np.linalg.norm(xa[:, :, None, :] - xb[:, None, :, :], axis=-1)
            j = np.argmin(d, axis=2)
            h = np.linalg.norm(xb[:, :, None, :] - xb[:, None, :, :], axis=-1)
            h = np.where(h == 0, np.inf, h).min(axis=(1, 2)) if nfpf > 1 else np.ones(len(j))
            dmin = np.take_along_axis(d, j[:, :, None], 2)[:, :, 0]
            if np.any(dmin > tol * np.maximum(h, 1e-300)[:, None] * 1e4):
                raise ValueError("flux points of a connected face do not coincide")
            for r in range(len(j)):
                e, fc, e2, fc2 = pe[c0 + r], pf[c0 + r], qe[c0 + r], qf[c0 + r]
                partner[e, fc * nfpf:(fc + 1) * nfpf] = e2 * nfp + fc2 * nfpf + j[r]

    for e in range(E):
        for fc in range(2 * dim):
            t = tags[e, fc]
            if t >= 2:
                bc[e, fc * nfpf:(fc + 1) * nfpf] = t
            elif partner[e, fc * nfpf] < 0:
                raise ValueError("face left unconnected")
    return partner, bc


def _face_points(mesh, ref, elems, faces):
    """Physical flux-point coordinates of face ``faces[i]`` of ``elems[i]``."""
    out = np.empty((len(elems), ref.nfpf, mesh.dim))
    nodes = mesh.node_coords()
    for fc in range(ref.nfaces):
        sel = np.nonzero(faces == fc)[0]
        if sel.size == 0:
            continue
        X = ref.fp_xi[fc * ref.nfpf:(fc + 1) * ref.nfpf]
        N, _ = _shape(mesh.geo_order, mesh.dim, X)
        out[sel] = np.einsum("pa,eaj->epj", N, nodes[elems[sel]])
    return out
