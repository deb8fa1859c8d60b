"""Compressible Navier-Stokes physics in FP64 (test infrastructure only).

Governing equations of Sec. 2.1 (Eqs. 1-7): du/dt + div F = 0 with
u = [rho, rho v_i, rho E], F = F_inv - F_vis,

  F_inv,j = [rho v_j, rho v_i v_j + delta_ij p, v_j (rho E + p)],
  p = (gamma - 1) rho (E - v_k v_k / 2),
  tau_ij = mu (dv_i/dx_j + dv_j/dx_i - 2/3 dv_k/dx_k delta_ij),
  q_j = -(mu / Pr) d/dx_j (E + p/rho - v_k v_k / 2).

Reading of the printed viscous energy flux: Eq. 4 prints
-q_j - v_i tau_ij; the physically consistent entry (viscous work enters with
a plus sign, heat flux with a minus sign, so that viscous dissipation heats
the fluid) is F_vis,j = [0, tau_ij, v_i tau_ij - q_j], which is used here.

Gradients are carried as grad[..., j, v] = d u_v / d x_j of the conserved
variables; velocity and energy gradients follow from the quotient rule.

Interface and boundary fluxes (the paper names the boundary types in
Secs. 3.1.1 and 4.1.1 but not their formulas; these are the readings used):

* Rusanov: F* n = 1/2 (F(u_L) + F(u_R)) . n - 1/2 lambda |n| (u_R - u_L),
  lambda = max over both sides of |v . n_hat| + c;
* Roe (alternative): Roe-averaged state, acoustic, entropy and shear waves,
  Harten's entropy fix (delta = 0.1 c) on the acoustic waves;
* no-slip adiabatic wall: inviscid ghost with mirrored velocity and the same
  density and pressure; wall state for gradients with zero velocity, the
  interior density and interior internal energy; viscous normal flux from
  the wall state with zero energy component;
* characteristic far field / inflow / outflow (subsonic): Riemann invariants
  R+ = v_n + 2c/(gamma-1) from the interior and R- = v_n - 2c/(gamma-1) from
  the reference state; tangential velocity and entropy from the interior when
  the boundary normal velocity points out of the domain, else from the
  reference state; inflow uses U tanh(3 (y - y_wall) / delta) along the free
  stream direction as the reference velocity.
"""
from __future__ import annotations

import numpy as np


class NavierStokes:
    def __init__(self, dim, gamma=1.4, mu=0.0, prandtl=0.71, viscous=False,
                 rho_inf=1.0, v_inf=None, p_inf=1.0, inflow_delta=0.0,
                 inflow_ywall=0.0, flux="rusanov"):
        self.dim = dim
        self.nvar = dim + 2
        self.gamma = gamma
        self.mu = mu
        self.prandtl = prandtl
        self.viscous = viscous
        self.rho_inf = rho_inf
        self.v_inf = np.zeros(dim) if v_inf is None else np.asarray(v_inf, float)
        self.p_inf = p_inf
        self.inflow_delta = inflow_delta
        self.inflow_ywall = inflow_ywall
        if flux not in ("rusanov", "roe"):
            raise ValueError(flux)
        self.flux = flux

    # -- primitive variables -------------------------------------------------
    def primitives(self, u):
        rho = u[..., 0]
        vel = u[..., 1:1 + self.dim] / rho[..., None]
        p = (self.gamma - 1.0) * (u[..., -1] - 0.5 * rho * np.sum(vel * vel, -1))
        return rho, vel, p

    def conserved(self, rho, vel, p):
        ke = 0.5 * rho * np.sum(vel * vel, -1)
        return np.concatenate([rho[..., None], rho[..., None] * vel,
                               (p / (self.gamma - 1.0) + ke)[..., None]], -1)

    def pressure(self, u):
        return self.primitives(u)[2]

    # -- fluxes -----------------------------------------------------------------
    def inviscid_flux(self, u):
        """F[..., j, v]."""
        rho, vel, p = self.primitives(u)
        d = self.dim
        F = np.empty(u.shape[:-1] + (d, self.nvar))
        for j in range(d):
            F[..., j, 0] = u[..., 1 + j]
            for i in range(d):
                F[..., j, 1 + i] = u[..., 1 + i] * vel[..., j] + (p if i == j else 0.0)
            F[..., j, -1] = vel[..., j] * (u[..., -1] + p)
        return F

    def viscous_flux(self, u, grad):
        """F_vis[..., j, v] from the state and conserved-variable gradients."""
        d = self.dim
        rho = u[..., 0]
        vel = u[..., 1:1 + d] / rho[..., None]
        Espec = u[..., -1] / rho
        grho = grad[..., :, 0]                                  # (..., j)
        gvel = (grad[..., :, 1:1 + d] - grho[..., :, None] * vel[..., None, :]) / rho[..., None, None]
        # gvel[..., j, i] = d v_i / d x_j
        gE = (grad[..., :, -1] - grho * Espec[..., None]) / rho[..., None]
        div = np.einsum("...ii->...", gvel)
        mu = self.mu
        tau = np.empty(u.shape[:-1] + (d, d))
        for i in range(d):
            for j in range(d):
                tau[..., i, j] = mu * (gvel[..., j, i] + gvel[..., i, j]
                                       - (2.0 / 3.0 * div if i == j else 0.0))
        # d/dx_j (E + p/rho - v.v/2) = gamma (dE/dx_j - v_k dv_k/dx_j)
        gh = self.gamma * (gE - np.einsum("...k,...jk->...j", vel, gvel))
        q = -(mu / self.prandtl) * gh
        F = np.zeros(u.shape[:-1] + (d, self.nvar))
        for j in range(d):
            for i in range(d):
                F[..., j, 1 + i] = tau[..., i, j]
            F[..., j, -1] = np.einsum("...i,...i->...", vel, tau[..., :, j]) - q[..., j]
        return F

    def sound_speed(self, rho, p):
        return np.sqrt(self.gamma * p / rho)

    def rusanov(self, uL, uR, n):
        """Common inviscid normal flux (outward normal n, scaled by |dS|)."""
        nmag = np.linalg.norm(n, axis=-1)
        nhat = n / nmag[..., None]
        FL = np.einsum("...jv,...j->...v", self.inviscid_flux(uL), n)
        FR = np.einsum("...jv,...j->...v", self.inviscid_flux(uR), n)
        rL, vL, pL = self.primitives(uL)
        rR, vR, pR = self.primitives(uR)
        lam = np.maximum(np.abs(np.sum(vL * nhat, -1)) + self.sound_speed(rL, pL),
                         np.abs(np.sum(vR * nhat, -1)) + self.sound_speed(rR, pR))
        return 0.5 * (FL + FR) - 0.5 * (lam * nmag)[..., None] * (uR - uL)

    def roe_waves(self, uL, uR, nhat):
        """Roe-averaged state and the wave decomposition of u_R - u_L along
        the unit normal: returns (lambdas, strengths, eigenvectors) with
        eigenvectors[..., k, :] the k-th right eigenvector (conserved
        variables).  Waves: v_n - c, v_n (entropy), v_n + c, and the shear
        jump (v_n; its 'strength' 1 and 'eigenvector' the shear vector)."""
        g1 = self.gamma - 1.0
        d = self.dim
        rL, vL, pL = self.primitives(uL)
        rR, vR, pR = self.primitives(uR)
        HL = (uL[..., -1] + pL) / rL
        HR = (uR[..., -1] + pR) / rR
        sL, sR = np.sqrt(rL), np.sqrt(rR)
        wL, wR = sL / (sL + sR), sR / (sL + sR)
        rt = sL * sR
        vt = wL[..., None] * vL + wR[..., None] * vR
        Ht = wL * HL + wR * HR
        q2 = np.sum(vt * vt, -1)
        ct = np.sqrt(g1 * (Ht - 0.5 * q2))
        vnt = np.sum(vt * nhat, -1)
        drho = rR - rL
        dp = pR - pL
        dv = vR - vL
        dvn = np.sum(dv * nhat, -1)
        dvt = dv - dvn[..., None] * nhat
        a1 = (dp - rt * ct * dvn) / (2 * ct * ct)
        a2 = drho - dp / (ct * ct)
        a3 = (dp + rt * ct * dvn) / (2 * ct * ct)
        shape = uL.shape[:-1]
        R = np.zeros(shape + (4, self.nvar))
        R[..., 0, 0] = 1.0
        R[..., 0, 1:1 + d] = vt - ct[..., None] * nhat
        R[..., 0, -1] = Ht - vnt * ct
        R[..., 1, 0] = 1.0
        R[..., 1, 1:1 + d] = vt
        R[..., 1, -1] = 0.5 * q2
        R[..., 2, 0] = 1.0
        R[..., 2, 1:1 + d] = vt + ct[..., None] * nhat
        R[..., 2, -1] = Ht + vnt * ct
        R[..., 3, 1:1 + d] = rt[..., None] * dvt
        R[..., 3, -1] = rt * np.sum(vt * dvt, -1)
        lam = np.stack([vnt - ct, vnt, vnt + ct, vnt], -1)
        alpha = np.stack([a1, a2, a3, np.ones_like(a1)], -1)
        return lam, alpha, R, ct

    def roe(self, uL, uR, n):
        """Roe's approximate Riemann solver (normal n scaled by |dS|):
        1/2 (F_L + F_R).n - 1/2 |n| sum_k |lambda_k| alpha_k r_k, with
        Harten's entropy fix on the two acoustic waves: |lambda| replaced by
        (lambda^2 + delta^2) / (2 delta) below delta = 0.1 c."""
        nmag = np.linalg.norm(n, axis=-1)
        nhat = n / nmag[..., None]
        FL = np.einsum("...jv,...j->...v", self.inviscid_flux(uL), n)
        FR = np.einsum("...jv,...j->...v", self.inviscid_flux(uR), n)
        lam, alpha, R, ct = self.roe_waves(uL, uR, nhat)
        alam = np.abs(lam)
        delta = 0.1 * ct
        for k in (0, 2):
            small = alam[..., k] < delta
            alam[..., k] = np.where(small, (lam[..., k] ** 2 + delta ** 2) / (2 * delta), alam[..., k])
        diss = np.einsum("...k,...kv->...v", alam * alpha, R)
        return 0.5 * (FL + FR) - 0.5 * nmag[..., None] * diss

    def common_inviscid(self, uL, uR, n):
        return self.roe(uL, uR, n) if self.flux == "roe" else self.rusanov(uL, uR, n)

    # -- boundary states ----------------------------------------------------------
    def wall_ghost(self, uL, nhat):
        """Mirror the velocity, keep density and pressure."""
        g = uL.copy()
        mn = np.sum(uL[..., 1:1 + self.dim] * nhat, -1)
        g[..., 1:1 + self.dim] = uL[..., 1:1 + self.dim] - 2.0 * mn[..., None] * nhat
        return g

    def wall_state(self, uL):
        """Zero velocity, interior density and internal energy."""
        rho, vel, p = self.primitives(uL)
        return self.conserved(rho, np.zeros_like(vel), p)

    def reference_velocity(self, tag, x):
        v = np.broadcast_to(self.v_inf, x.shape[:-1] + (self.dim,)).copy()
        if tag == 4 and self.inflow_delta > 0.0:
            prof = np.tanh(3.0 * (x[..., 1] - self.inflow_ywall) / self.inflow_delta)
            v = v * prof[..., None]
        return v

    def riemann_state(self, uL, nhat, v_ref):
        g1 = self.gamma - 1.0
        rL, vL, pL = self.primitives(uL)
        cL = self.sound_speed(rL, pL)
        c_inf = np.sqrt(self.gamma * self.p_inf / self.rho_inf)
        vnL = np.sum(vL * nhat, -1)
        vn_ref = np.sum(v_ref * nhat, -1)
        Rp = vnL + 2.0 * cL / g1
        Rm = vn_ref - 2.0 * c_inf / g1
        vnb = 0.5 * (Rp + Rm)
        cb = 0.25 * g1 * (Rp - Rm)
        out = vnb > 0.0
        s_in = pL / rL ** self.gamma
        s_ref = self.p_inf / self.rho_inf ** self.gamma
        s = np.where(out, s_in, s_ref)
        vt = np.where(out[..., None], vL - vnL[..., None] * nhat,
                      v_ref - vn_ref[..., None] * nhat)
        vb = vt + vnb[..., None] * nhat
        rb = (cb * cb / (self.gamma * s)) ** (1.0 / g1)
        pb = rb * cb * cb / self.gamma
        return self.conserved(rb, vb, pb)

    def boundary_states(self, tag, uL, n, x):
        """(ghost for the inviscid flux, state for gradients) at boundary
        flux points of one tag."""
        nhat = n / np.linalg.norm(n, axis=-1)[..., None]
        if tag == 2:
            return self.wall_ghost(uL, nhat), self.wall_state(uL)
        ub = self.riemann_state(uL, nhat, self.reference_velocity(tag, x))
        return ub, ub

    def boundary_viscous_flux(self, tag, ub, Q, n):
        """Common viscous normal flux at boundary points."""
        fv = np.einsum("...jv,...j->...v", self.viscous_flux(ub, Q), n)
        if tag == 2:
            fv[..., -1] = 0.0
        return fv


class ScalarDiffusion:
    """u_t = div(nu grad u), written as du/dt + div F = 0 with F_inv = 0 and
    F_vis = nu grad u; periodic meshes only.  Used to pin the gradient,
    lifting and viscous-flux machinery against exact heat-equation decay."""

    def __init__(self, dim, nu):
        self.dim = dim
        self.nvar = 1
        self.nu = nu
        self.viscous = True

    def inviscid_flux(self, u):
        return np.zeros(u.shape[:-1] + (self.dim, 1))

    def viscous_flux(self, u, grad):
        return self.nu * grad

    def rusanov(self, uL, uR, n):
        return np.zeros_like(uL)

    def common_inviscid(self, uL, uR, n):
        return np.zeros_like(uL)
