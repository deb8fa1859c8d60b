"""FR residual du/dt at the solution points, FP64, plain dense operators
(test infrastructure only; never imported by the product path).

The paper's spatial discretisation is Huynh's Flux Reconstruction (Sec. 2.3)
with details deferred to its references; the steps below are the textbook
scheme with the choices named in the module docstrings of ``element``,
``geometry`` and ``physics``:

1. u_f = M0 u: solution at the flux points.
2. (viscous) u_c = (u_L + u_R)/2 on interior/periodic points, the boundary
   state on boundary points; corrected reference gradient
   G_k = D_k u + Cgrad_k (u_c - u_f); physical gradient
   grad_j = (1/J) sum_k S[k, j] G_k.
3. (viscous, BR2) face gradient Q_f = interp_f((1/J) S^T D u) + eta r_f,
   where r_f is the lifting of face f's own jump alone, evaluated at f;
   common viscous normal flux 1/2 (F_vis(u_L, Q_L) + F_vis(u_R, Q_R)) . n.
4. Transformed flux at solution points F^k = sum_j S[k, j] F_j with
   F = F_inv(u) - F_vis(u, grad).
5. Discontinuous normal flux at a flux point: sign * (M0 F^k)_f, the value of
   the flux polynomial along the line (Huynh's f^D at the element edge).
6. Jump = common normal flux (Rusanov - viscous common) - discontinuous.
7. div = sum_k D_k F^k + Cdiv jump; du/dt = -div / J.

``residual`` can evaluate a subset of elements: it then works on the one-
(inviscid) or two-ring (viscous) neighbourhood of that subset only.
"""
from __future__ import annotations

import numpy as np

from .element import RefElement
from .geometry import Geometry, connectivity


class FRDiscretisation:
    """``viscous_scheme``: "br2" (default) or "ldg".  LDG reading: every
    interface has a fixed left side, the side whose flux point has the
    smaller index (element * nfp + point); with s = +1 there and -1 on the
    other side, the common solution is (1/2 + s beta) u_own + (1/2 - s beta)
    u_other, the face gradient is the corrected gradient interpolated to the
    face (no lifting), and the common viscous normal flux is
    (1/2 - s beta) F_v,own . n + (1/2 + s beta) F_v,other . n
    - tau |n| (u_own - u_other); boundary points as for BR2."""

    def __init__(self, mesh, p, phys, br2_eta=None, viscous_scheme="br2", ldg_beta=0.5,
                 ldg_tau=0.1):
        self.mesh = mesh
        self.ref = RefElement(mesh.dim, p)
        self.phys = phys
        self.partner, self.bc = connectivity(mesh, self.ref)
        nfp = self.ref.nfp
        self.partner_elem = np.where(self.partner >= 0, self.partner // nfp, -1)
        self.eta = float(2 * mesh.dim if br2_eta is None or br2_eta <= 0 else br2_eta)
        if viscous_scheme not in ("br2", "ldg"):
            raise ValueError(viscous_scheme)
        self.scheme = viscous_scheme
        self.beta, self.tau = ldg_beta, ldg_tau
        own = np.arange(mesh.n_elem)[:, None] * nfp + np.arange(nfp)[None, :]
        self.side = np.where(own < self.partner, 1.0, -1.0)     # +1 on an interface's left side
        self._geo_all = None

    # -- geometry ---------------------------------------------------------------
    def geometry(self, elems=None):
        if elems is None:
            if self._geo_all is None:
                self._geo_all = Geometry(self.mesh, self.ref, np.arange(self.mesh.n_elem))
            return self._geo_all
        return Geometry(self.mesh, self.ref, elems)

    def sol_coords(self):
        return self.geometry().x_sp

    def _ring(self, elems):
        nb = self.partner_elem[elems].ravel()
        nb = nb[nb >= 0]
        return np.union1d(elems, nb)

    # -- pieces shared by the residual and the wall force ---------------------------
    def _outer_state(self, ctx, set_):
        """(u_L, u_R, boundary state, tags) at all flux points of set_."""
        loc, geoC, UC, Uf = ctx
        phys, nfp = self.phys, self.ref.nfp
        rows = loc[set_]
        part = self.partner[set_]
        pe = np.where(part >= 0, part // nfp, 0)
        pf = np.where(part >= 0, part % nfp, 0)
        uR = Uf[loc[pe], pf]
        uL = Uf[rows]
        uB = uR.copy()
        bcs = self.bc[set_]
        for tag in (2, 3, 4, 5):
            m = bcs == tag
            if np.any(m):
                g, b = phys.boundary_states(tag, uL[m], geoC.n[rows][m], geoC.x_fp[rows][m])
                uR[m] = g
                uB[m] = b
        return uL, uR, uB, bcs

    def _viscous_faces(self, ctx, B):
        """Steps 2-3 for the elements B: corrected gradient at the solution
        points and the viscous normal flux at their flux points (own side on
        connected points, the common flux on boundary points)."""
        loc, geoC, UC, Uf = ctx
        ref, phys = self.ref, self.phys
        nfp = ref.nfp
        rowsB = loc[B]
        uLB, uRB, uBB, bcsB = self._outer_state(ctx, B)
        if self.scheme == "ldg":
            bs = (self.beta * self.side[B])[..., None]
            uc_int = (0.5 + bs) * uLB + (0.5 - bs) * uRB
        else:
            uc_int = 0.5 * (uLB + uRB)
        uc = np.where((bcsB > 0)[..., None], uBB, uc_int)
        dU = uc - uLB                                                # (nB, nfp, V)
        SB, JB = geoC.S[rowsB], geoC.J[rowsB]
        Du = np.einsum("kst,etv->eskv", ref.D, UC[rowsB])            # D_k u
        G = Du + np.einsum("ksf,efv->eskv", ref.Cgrad, dU)           # step 2
        grad = np.einsum("eskj,eskv->esjv", SB, G) / JB[..., None, None]
        gradD = np.einsum("eskj,eskv->esjv", SB, Du) / JB[..., None, None]
        # step 3: BR2 face gradient Q = interp(grad^D) + eta r_f, with
        # r_f[j] = sum_s M0[f,s] Cgrad[k_f][s,f] S[s,k_f,j] / J[s] * dU_f
        Qd = np.einsum("fs,esjv->efjv", ref.M0, gradD)
        kf = ref.fp_dir
        Cg = ref.Cgrad[kf, :, np.arange(nfp)]                        # (nfp, nsp)
        W = ref.M0 * Cg
        Lf = np.empty((len(B), nfp, self.mesh.dim))
        for k in range(self.mesh.dim):
            fk = kf == k
            Lf[:, fk, :] = np.einsum("fs,esj->efj", W[fk], SB[:, :, k, :] / JB[:, :, None])
        Q = Qd + self.eta * Lf[..., :, None] * dU[..., None, :]
        if self.scheme == "ldg":
            Q = np.einsum("fs,esjv->efjv", ref.M0, grad)             # corrected, no lifting
        nB = geoC.n[rowsB]
        fv_own = np.einsum("efjv,efj->efv", phys.viscous_flux(uLB, Q), nB)
        for tag in (2, 3, 4, 5):
            m = bcsB == tag
            if np.any(m):
                fv_own[m] = phys.boundary_viscous_flux(tag, uBB[m], Q[m], nB[m])
        return grad, fv_own, uLB, uBB, bcsB, nB

    def wall_force(self, U):
        """Force of the fluid on all wall faces, sum over wall flux points of
        w_f (p n - tau . n) with n the fluid's outward normal scaled by the
        surface Jacobian (Sec. 3.1.2 uses the wall force for C_D)."""
        ref, phys = self.ref, self.phys
        E = self.mesh.n_elem
        B = np.nonzero(np.any(self.bc == 2, axis=1))[0]
        F = np.zeros(self.mesh.dim)
        if B.size == 0:
            return F
        C = self._ring(B)
        loc = np.full(E, -1, dtype=np.int64)
        loc[C] = np.arange(C.size)
        geoC = self.geometry(C)
        UC = U[C]
        Uf = np.einsum("fs,esv->efv", ref.M0, UC)
        ctx = (loc, geoC, UC, Uf)
        uL, _, _, bcs = self._outer_state(ctx, B)
        nB = geoC.n[loc[B]]
        m = bcs == 2
        p = phys.pressure(uL)
        wgt = np.broadcast_to(ref.fp_w, bcs.shape)
        F += np.einsum("i,ij->j", (wgt * p)[m], nB[m])
        if phys.viscous:
            _, fv, _, _, _, _ = self._viscous_faces(ctx, B)
            F -= np.einsum("i,ij->j", wgt[m], fv[m][:, 1:1 + self.mesh.dim])
        return F

    # -- residual -------------------------------------------------------------------
    def residual(self, U, elems=None, magnitude=False):
        """du/dt at the solution points of ``elems`` (all when None).

        With ``magnitude=True`` it also returns the sum of the absolute values
        of the terms that step 7 adds up, divided by J: the scale of the
        floating-point error bound of the residual (a sum of n terms computed
        in precision eps has error at most about n eps times this)."""
        ref, phys = self.ref, self.phys
        E = self.mesh.n_elem
        if elems is None:
            A = np.arange(E)
            B = C = A
        else:
            A = np.unique(np.asarray(elems, dtype=np.int64))
            B = self._ring(A)
            C = self._ring(B) if phys.viscous else B
        loc = np.full(E, -1, dtype=np.int64)
        loc[C] = np.arange(C.size)
        geoC = self.geometry() if elems is None else self.geometry(C)
        nfp = ref.nfp

        UC = U[C]
        Uf = np.einsum("fs,esv->efv", ref.M0, UC)                  # step 1
        ctx = (loc, geoC, UC, Uf)

        if phys.viscous:
            grad, fv_own, _, _, _, _ = self._viscous_faces(ctx, B)
            locB = np.full(E, -1, dtype=np.int64)
            locB[B] = np.arange(B.size)
            gradA = grad[locB[A]]
            fvA = fv_own[locB[A]]
        rowsA = loc[A]
        uLA, uRA, _, bcsA = self._outer_state(ctx, A)
        SA, JA, nA = geoC.S[rowsA], geoC.J[rowsA], geoC.n[rowsA]
        F = phys.inviscid_flux(UC[rowsA])                            # (nA, nsp, d, V)
        if phys.viscous:
            F = F - phys.viscous_flux(UC[rowsA], gradA)
        Fhat = np.einsum("eskj,esjv->eskv", SA, F)                   # step 4
        kf = ref.fp_dir
        Fdisc = np.empty(uLA.shape)                                  # step 5
        for k in range(self.mesh.dim):
            fk = kf == k
            Fdisc[:, fk, :] = np.einsum("fs,esv->efv", ref.M0[fk], Fhat[:, :, k, :])
        Fdisc *= ref.fp_sign[None, :, None]
        Fstar = phys.common_inviscid(uLA, uRA, nA)
        if phys.viscous:
            part = self.partner[A]
            pe = np.where(part >= 0, part // nfp, 0)
            pf = np.where(part >= 0, part % nfp, 0)
            fvR = fv_own[locB[pe], pf]
            if self.scheme == "ldg":
                bs = (self.beta * self.side[A])[..., None]
                nmag = np.linalg.norm(nA, axis=-1)[..., None]
                interior = (0.5 - bs) * fvA - (0.5 + bs) * fvR - self.tau * nmag * (uLA - uRA)
            else:
                interior = 0.5 * (fvA - fvR)
            fv_common = np.where((bcsA > 0)[..., None], fvA, interior)
            Fstar = Fstar - fv_common
        jump = Fstar - Fdisc                                         # step 6
        div = np.einsum("kst,etkv->esv", ref.D, Fhat) + np.einsum("sf,efv->esv", ref.Cdiv, jump)
        if magnitude:
            mag = (np.einsum("kst,etkv->esv", np.abs(ref.D), np.abs(Fhat))
                   + np.einsum("sf,efv->esv", np.abs(ref.Cdiv), np.abs(Fstar) + np.abs(Fdisc)))
            return -div / JA[..., None], mag / JA[..., None]
        return -div / JA[..., None]                                  # step 7
