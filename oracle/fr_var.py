"""FR residual with a solution degree chosen per element, FP64 (test
infrastructure only; never imported by the product path).

Sec. 5.1 runs the airfoil grids with a variable solution degree (P0-P3 and
P0-P4 distributions): the outer zones carry low degrees so that the waves are
damped before they reach the boundaries.  The paper does not say how a face
between two elements of different degree is treated.  The reading taken here
is the mortar element method (Kopriva, 1996), the usual conservative
coupling of tensor-product spectral elements of unequal degree:

* a face joining two elements of the same degree is treated as in ``fr``;
* on a face joining degrees p_lo < p_hi the mortar is the higher side's set
  of flux points.  The lower side's face trace (a polynomial of degree p_lo
  in the face coordinates) is evaluated there (operator T); the higher
  side's trace reaches the lower side as its L2 projection onto degree p_lo
  in the face's reference coordinates (operator P);
* the common solution of BR2 / LDG on each side is formed from its own trace
  and the partner's trace carried to its own points; being linear in the
  traces, the lower side's common solution is the projection of the mortar's;
* the common normal flux is formed at the mortar points: the inviscid flux
  from the higher side's trace and the lower side's trace carried there by
  T, the viscous part from the higher side's own viscous normal flux and the
  lower side's own viscous normal flux carried there by T.  The higher side
  uses it as it is; the lower side receives minus its L2 projection (the
  outward normals are opposite).  The projection keeps the face integral of
  the flux, so the scheme stays conservative;
* LDG's one-sided switch: on such a face the lower-degree side is the left
  side; on other faces the side with the smaller (element, flux point) pair,
  as in ``fr``.

T is built by locating each mortar point in the lower element with Newton's
method; P from its definition, M P = B with M and B the face mass and mixed
mass matrices integrated by an 8-point Gauss rule per direction (exact for
the degrees involved).

State layout: one flat array (sum over elements of (p_e + 1)^dim, V),
element after element, each element's points in its reference element's
order.
"""
from __future__ import annotations

import numpy as np

from . import basis
from .element import RefElement
from .geometry import Geometry, face_pairs, map_points, jacobian
from .acoustics import locate as _locate_in_mesh


def locate_in(mesh, e, X, tol=1e-14, max_iter=50):
    """Reference coordinates in element ``e`` of the physical points X
    (npts, dim), by Newton's method on the element map."""
    X = np.atleast_2d(np.asarray(X, float))
    xi = np.zeros_like(X)
    for _ in range(max_iter):
        x = map_points(mesh, [e], xi)[0]
        A = jacobian(mesh, [e], xi)[0]
        dxi = np.linalg.solve(A, (X - x)[..., None])[..., 0]
        xi = xi + dxi
        if np.max(np.abs(dxi)) < tol:
            break
    return xi


def free_dirs(dim, face):
    k = face // 2
    return [a for a in range(dim) if a != k]


def face_basis(ref, sigma):
    """Lagrange basis of one face's flux points (tensor product of the 1-D
    Gauss nodes, lower free direction fastest) at face coordinates sigma
    (npts, dim - 1): returns (npts, nfpf)."""
    sigma = np.atleast_2d(sigma)
    out = np.ones((sigma.shape[0], ref.nfpf))
    for a in range(ref.dim - 1):
        La = basis.lagrange(ref.xi, sigma[:, a])
        idx = (np.arange(ref.nfpf) // ref.n ** a) % ref.n
        out *= La[:, idx]
    return out


def _face_xi(dim, face, sigma):
    """Element reference coordinates of face coordinates sigma on ``face``."""
    sigma = np.atleast_2d(sigma)
    xi = np.empty((sigma.shape[0], dim))
    k = face // 2
    xi[:, k] = 1.0 if face % 2 else -1.0
    xi[:, free_dirs(dim, face)] = sigma
    return xi


def _partner_face_coords(mesh, e, face, e2, face2, shift, sigma, tol=1e-9):
    """Face coordinates on (e2, face2) of the points with face coordinates
    sigma on (e, face)."""
    x = map_points(mesh, [e], _face_xi(mesh.dim, face, sigma))[0] + shift
    xi2 = locate_in(mesh, e2, x)
    k2 = face2 // 2
    on = 1.0 if face2 % 2 else -1.0
    if np.max(np.abs(xi2[:, k2] - on)) > tol or np.max(np.abs(xi2)) > 1.0 + tol:
        raise ValueError("points of a connected face do not lie on the partner face")
    return xi2[:, free_dirs(mesh.dim, face2)]


def transfer_matrix(mesh, refs, e, face, e2, face2, shift):
    """T (nfpf_own, nfpf_partner): the partner's face polynomial evaluated at
    this face's flux points."""
    r = refs[e]
    sigma = r.fp_xi[face * r.nfpf:(face + 1) * r.nfpf][:, free_dirs(mesh.dim, face)]
    sigma2 = _partner_face_coords(mesh, e, face, e2, face2, shift, sigma)
    return face_basis(refs[e2], sigma2)


def projection_matrix(mesh, refs, e, face, e2, face2, shift, nq=8):
    """P (nfpf_own, nfpf_partner): L2 projection, in this face's reference
    coordinates, of the partner's face polynomial onto this side's degree:
    M P = B, M_ik = int l_i l_k, B_ij = int l_i L_j(partner coords)."""
    dim = mesh.dim
    xq, wq = basis.gauss_legendre(nq)
    if dim == 2:
        sig = xq[:, None]
        W = wq
    else:
        sig = np.stack([np.tile(xq, nq), np.repeat(xq, nq)], axis=1)
        W = np.tile(wq, nq) * np.repeat(wq, nq)
    Lo = face_basis(refs[e], sig)                                        # (nq^, own)
    Lp = face_basis(refs[e2], _partner_face_coords(mesh, e, face, e2, face2, shift, sig))
    M = np.einsum("q,qi,qk->ik", W, Lo, Lo)
    B = np.einsum("q,qi,qj->ij", W, Lo, Lp)
    return np.linalg.solve(M, B)


class VarFRDiscretisation:
    """FR residual du/dt on a mesh whose element e has degree elem_p[e]
    (0..4 in the tests; the operators are defined for any degree >= 0)."""

    def __init__(self, mesh, elem_p, phys, br2_eta=None, viscous_scheme="br2", ldg_beta=0.5,
                 ldg_tau=0.1):
        self.mesh, self.phys = mesh, phys
        dim, E = mesh.dim, mesh.n_elem
        self.elem_p = np.asarray(elem_p, dtype=np.int64)
        if self.elem_p.shape != (E,):
            raise ValueError("one degree per element")
        self.degrees = sorted(set(int(q) for q in self.elem_p))
        self.refq = {q: RefElement(dim, q) for q in self.degrees}
        self.refs = [self.refq[int(q)] for q in self.elem_p]
        self.members = {q: np.nonzero(self.elem_p == q)[0] for q in self.degrees}
        self.loc = np.empty(E, dtype=np.int64)
        for q in self.degrees:
            self.loc[self.members[q]] = np.arange(self.members[q].size)
        self.geo = {q: Geometry(mesh, self.refq[q], self.members[q]) for q in self.degrees}
        self.eta = float(2 * dim if br2_eta is None or br2_eta <= 0 else br2_eta)
        if viscous_scheme not in ("br2", "ldg"):
            raise ValueError(viscous_scheme)
        self.scheme = viscous_scheme
        self.beta, self.tau = ldg_beta, ldg_tau
        nsp_e = np.array([r.nsp for r in self.refs])
        self.sp_off = np.concatenate([[0], np.cumsum(nsp_e)])
        self.n_sp = int(self.sp_off[-1])
        self.sp_index = {q: self.sp_off[self.members[q]][:, None] + np.arange(self.refq[q].nsp)[None, :]
                         for q in self.degrees}

        # connections, seen from each side: (e, face) -> link
        self.links = {}
        for (e, fc, e2, fc2, sh) in face_pairs(mesh):
            r, r2 = self.refs[e], self.refs[e2]
            if r.p == r2.p:
                xa = self.geo[r.p].x_fp[self.loc[e], fc * r.nfpf:(fc + 1) * r.nfpf] + sh
                xb = self.geo[r.p].x_fp[self.loc[e2], fc2 * r.nfpf:(fc2 + 1) * r.nfpf]
                d = np.linalg.norm(xa[:, None, :] - xb[None, :, :], axis=-1)
                j = np.argmin(d, axis=1)
                h = np.linalg.norm(xb[:, None] - xb[None, :], axis=-1)
                h = h[h > 0].min() if r.nfpf > 1 else 1.0
                if np.max(d[np.arange(r.nfpf), j]) > 1e-6 * h:
                    raise ValueError("flux points of a connected face do not coincide")
                self.links[(e, fc)] = ("same", e2, fc2, j)
            elif r.p > r2.p:
                self.links[(e, fc)] = ("hi", e2, fc2, transfer_matrix(mesh, self.refs, e, fc, e2, fc2, sh))
            else:
                self.links[(e, fc)] = ("lo", e2, fc2, projection_matrix(mesh, self.refs, e, fc, e2, fc2, sh))
        for e in range(E):
            for fc in range(2 * dim):
                if mesh.face_tag[e, fc] < 2 and (e, fc) not in self.links:
                    raise ValueError("face left unconnected")

        # per degree: boundary tags and LDG sides at the flux points
        self.bc, self.side = {}, {}
        for q in self.degrees:
            r = self.refq[q]
            n_q = self.members[q].size
            self.bc[q] = np.zeros((n_q, r.nfp), dtype=np.int32)
            self.side[q] = np.zeros((n_q, r.nfp))
            for le, e in enumerate(self.members[q]):
                for fc in range(2 * dim):
                    rows = slice(fc * r.nfpf, (fc + 1) * r.nfpf)
                    t = mesh.face_tag[e, fc]
                    if t >= 2:
                        self.bc[q][le, rows] = t
                        continue
                    kind, e2, fc2, X = self.links[(e, fc)]
                    if kind == "same":
                        own = np.arange(fc * r.nfpf, (fc + 1) * r.nfpf)
                        oth = fc2 * r.nfpf + X
                        left = (e < e2) | ((e == e2) & (own < oth))
                        self.side[q][le, rows] = np.where(left, 1.0, -1.0)
                    else:
                        self.side[q][le, rows] = 1.0 if kind == "lo" else -1.0

    # -- layout helpers -------------------------------------------------------------
    def blocks(self, U):
        return {q: U[self.sp_index[q]] for q in self.degrees}

    def flat(self, blocks):
        V = next(iter(blocks.values())).shape[-1]
        out = np.empty((self.n_sp, V))
        for q in self.degrees:
            out[self.sp_index[q]] = blocks[q]
        return out

    def sol_coords(self):
        return self.flat({q: self.geo[q].x_sp for q in self.degrees})

    # -- face traces ------------------------------------------------------------------
    def _partner_traces(self, Uf):
        """Partner trace at every own flux point (boundary points: the ghost),
        the boundary state, and the face rows of each link."""
        mesh, phys = self.mesh, self.phys
        uR = {q: np.zeros_like(Uf[q]) for q in self.degrees}
        uB = {q: np.zeros_like(Uf[q]) for q in self.degrees}
        for (e, fc), (kind, e2, fc2, X) in self.links.items():
            q, q2 = int(self.elem_p[e]), int(self.elem_p[e2])
            r, r2 = self.refq[q], self.refq[q2]
            rows = slice(fc * r.nfpf, (fc + 1) * r.nfpf)
            rows2 = slice(fc2 * r2.nfpf, (fc2 + 1) * r2.nfpf)
            if kind == "same":
                uR[q][self.loc[e], rows] = Uf[q2][self.loc[e2], fc2 * r2.nfpf + X]
            else:
                uR[q][self.loc[e], rows] = X @ Uf[q2][self.loc[e2], rows2]
        for q in self.degrees:
            g = self.geo[q]
            for tag in (2, 3, 4, 5):
                m = self.bc[q] == tag
                if np.any(m):
                    gh, b = phys.boundary_states(tag, Uf[q][m], g.n[m], g.x_fp[m])
                    uR[q][m] = gh
                    uB[q][m] = b
        return uR, uB

    def _viscous(self, Ub, Uf, uR, uB):
        """Corrected gradient at the solution points and own-side viscous
        normal flux at the flux points (common flux at boundary points),
        per degree: the same steps as ``fr``."""
        phys, dim = self.phys, self.mesh.dim
        grad, fv = {}, {}
        for q in self.degrees:
            r, g = self.refq[q], self.geo[q]
            uL, bcs = Uf[q], self.bc[q]
            if self.scheme == "ldg":
                bs = (self.beta * self.side[q])[..., None]
                uc_int = (0.5 + bs) * uL + (0.5 - bs) * uR[q]
            else:
                uc_int = 0.5 * (uL + uR[q])
            uc = np.where((bcs > 0)[..., None], uB[q], uc_int)
            dU = uc - uL
            S, J = g.S, g.J
            Du = np.einsum("kst,etv->eskv", r.D, Ub[q])
            G = Du + np.einsum("ksf,efv->eskv", r.Cgrad, dU)
            grad[q] = np.einsum("eskj,eskv->esjv", S, G) / J[..., None, None]
            if self.scheme == "ldg":
                Q = np.einsum("fs,esjv->efjv", r.M0, grad[q])
            else:
                gradD = np.einsum("eskj,eskv->esjv", S, Du) / J[..., None, None]
                Qd = np.einsum("fs,esjv->efjv", r.M0, gradD)
                kf = r.fp_dir
                W = r.M0 * r.Cgrad[kf, :, np.arange(r.nfp)]
                Lf = np.empty((S.shape[0], r.nfp, dim))
                for k in range(dim):
                    fk = kf == k
                    Lf[:, fk, :] = np.einsum("fs,esj->efj", W[fk], S[:, :, k, :] / J[:, :, None])
                Q = Qd + self.eta * Lf[..., :, None] * dU[..., None, :]
            f = np.einsum("efjv,efj->efv", phys.viscous_flux(uL, Q), g.n)
            for tag in (2, 3, 4, 5):
                m = bcs == tag
                if np.any(m):
                    f[m] = phys.boundary_viscous_flux(tag, uB[q][m], Q[m], g.n[m])
            fv[q] = f
        return grad, fv

    # -- residual -------------------------------------------------------------------
    def residual(self, U, magnitude=False):
        """du/dt at every solution point (flat layout).  With
        ``magnitude=True`` also the sum of the absolute values of the terms
        of the divergence, divided by J (the scale of the rounding bound)."""
        phys, dim = self.phys, self.mesh.dim
        Ub = self.blocks(U)
        Uf = {q: np.einsum("fs,esv->efv", self.refq[q].M0, Ub[q]) for q in self.degrees}
        uR, uB = self._partner_traces(Uf)
        if phys.viscous:
            grad, fv = self._viscous(Ub, Uf, uR, uB)
        Fhat, Fdisc, Fstar = {}, {}, {}
        for q in self.degrees:
            r, g = self.refq[q], self.geo[q]
            F = phys.inviscid_flux(Ub[q])
            if phys.viscous:
                F = F - phys.viscous_flux(Ub[q], grad[q])
            Fhat[q] = np.einsum("eskj,esjv->eskv", g.S, F)
            fd = np.empty(Uf[q].shape)
            for k in range(dim):
                fk = r.fp_dir == k
                fd[:, fk, :] = np.einsum("fs,esv->efv", r.M0[fk], Fhat[q][:, :, k, :])
            Fdisc[q] = fd * r.fp_sign[None, :, None]
            Fstar[q] = phys.common_inviscid(Uf[q], uR[q], g.n)
        if phys.viscous:
            # partner's own viscous normal flux at the own points (same degree:
            # the paired point; higher side of a mortar: carried by T)
            fvR = {q: np.zeros_like(fv[q]) for q in self.degrees}
            for (e, fc), (kind, e2, fc2, X) in self.links.items():
                q, q2 = int(self.elem_p[e]), int(self.elem_p[e2])
                r, r2 = self.refq[q], self.refq[q2]
                rows = slice(fc * r.nfpf, (fc + 1) * r.nfpf)
                if kind == "same":
                    fvR[q][self.loc[e], rows] = fv[q2][self.loc[e2], fc2 * r2.nfpf + X]
                elif kind == "hi":
                    fvR[q][self.loc[e], rows] = X @ fv[q2][self.loc[e2], fc2 * r2.nfpf:(fc2 + 1) * r2.nfpf]
            for q in self.degrees:
                g = self.geo[q]
                if self.scheme == "ldg":
                    bs = (self.beta * self.side[q])[..., None]
                    nmag = np.linalg.norm(g.n, axis=-1)[..., None]
                    interior = ((0.5 - bs) * fv[q] - (0.5 + bs) * fvR[q]
                                - self.tau * nmag * (Uf[q] - uR[q]))
                else:
                    interior = 0.5 * (fv[q] - fvR[q])
                Fstar[q] = Fstar[q] - np.where((self.bc[q] > 0)[..., None], fv[q], interior)
        # lower side of a mortar: minus the projection of the higher side's flux
        Fmag = {q: np.abs(Fstar[q]) for q in self.degrees}
        for (e, fc), (kind, e2, fc2, X) in self.links.items():
            if kind != "lo":
                continue
            q, q2 = int(self.elem_p[e]), int(self.elem_p[e2])
            r, r2 = self.refq[q], self.refq[q2]
            rows = slice(fc * r.nfpf, (fc + 1) * r.nfpf)
            hi = Fstar[q2][self.loc[e2], fc2 * r2.nfpf:(fc2 + 1) * r2.nfpf]
            Fstar[q][self.loc[e], rows] = -(X @ hi)
            Fmag[q][self.loc[e], rows] = np.abs(X) @ np.abs(hi)
        out, mag = {}, {}
        for q in self.degrees:
            r, g = self.refq[q], self.geo[q]
            jump = Fstar[q] - Fdisc[q]
            div = (np.einsum("kst,etkv->esv", r.D, Fhat[q])
                   + np.einsum("sf,efv->esv", r.Cdiv, jump))
            out[q] = -div / g.J[..., None]
            if magnitude:
                m = (np.einsum("kst,etkv->esv", np.abs(r.D), np.abs(Fhat[q]))
                     + np.einsum("sf,efv->esv", np.abs(r.Cdiv), Fmag[q] + np.abs(Fdisc[q])))
                mag[q] = m / g.J[..., None]
        if magnitude:
            return self.flat(out), self.flat(mag)
        return self.flat(out)

    # -- observers --------------------------------------------------------------------
    def wall_force(self, U):
        """Force of the fluid on the wall faces: sum over wall flux points of
        w_f (p n - tau . n), as in ``fr``."""
        phys = self.phys
        F = np.zeros(self.mesh.dim)
        Ub = self.blocks(U)
        Uf = {q: np.einsum("fs,esv->efv", self.refq[q].M0, Ub[q]) for q in self.degrees}
        if phys.viscous:
            uR, uB = self._partner_traces(Uf)
            _, fv = self._viscous(Ub, Uf, uR, uB)
        for q in self.degrees:
            r, g = self.refq[q], self.geo[q]
            m = self.bc[q] == 2
            if not np.any(m):
                continue
            wgt = np.broadcast_to(r.fp_w, m.shape)
            F += np.einsum("i,ij->j", (wgt * phys.pressure(Uf[q]))[m], g.n[m])
            if phys.viscous:
                F -= np.einsum("i,ij->j", wgt[m], fv[q][m][:, 1:1 + self.mesh.dim])
        return F

    def integral(self, U):
        """sum over elements and solution points of w J U (per variable)."""
        Ub = self.blocks(U)
        tot = 0.0
        for q in self.degrees:
            tot = tot + np.einsum("s,es,esv->v", self.refq[q].sp_w, self.geo[q].J, Ub[q])
        return tot

    def probe_state(self, U, x_obs):
        """Conserved state at a physical point: the containing element's
        tensor Lagrange interpolant."""
        e, xi = _locate_in_mesh(self.mesh, None, x_obs)
        w = self.refs[e].interp_matrix(xi[None, :])[0]
        return w @ U[self.sp_off[e]:self.sp_off[e + 1]]
