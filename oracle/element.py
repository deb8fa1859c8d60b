"""Tensor-product FR reference element (quadrilateral or hexahedron), FP64.

Test infrastructure only.

Point sets and numbering (the reading of the FR scheme of Sec. 2.3 that this
code and the CUDA library both follow):

* solution points: the tensor product of the n = p+1 Gauss-Legendre nodes,
  index s = i + n j (+ n^2 k), xi index fastest;
* flux points: on each face the tensor product of the same 1-D nodes, faces
  ordered -xi, +xi, -eta, +eta (, -zeta, +zeta), points within a face
  ordered with the lower-numbered free direction fastest; index
  f = face * n^(d-1) + local;
* every flux point sits at the end of one line of n solution points running
  along the face-normal reference direction.

Dense operators (plain definitions, applied per element with a matmul):

* M0  (nfp x nsp): value at the flux point of the degree-p Lagrange
  interpolant along its line;
* D[k] (nsp x nsp): derivative along reference direction k;
* Cdiv (nsp x nfp): maps outward normal flux jumps at the flux points to the
  divergence correction, +g_R' for a + face, -g_L' for a - face (the - face's
  outward normal points along -xi^k);
* Cgrad[k] (nsp x nfp): maps solution jumps u_c - u_f on the two faces normal
  to k to the correction of d u / d xi^k, g_R' for +, g_L' for -.
"""
from __future__ import annotations

import itertools
import numpy as np

from . import basis


class RefElement:
    def __init__(self, dim: int, p: int):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim, self.p = dim, p
        n = p + 1
        self.n = n
        self.xi, self.w = basis.gauss_legendre(n)
        self.nsp = n ** dim
        self.nfpf = n ** (dim - 1)
        self.nfp = 2 * dim * self.nfpf
        self.nfaces = 2 * dim

        # multi-indices of solution points, direction 0 fastest
        self.sp_idx = np.array([t[::-1] for t in itertools.product(range(n), repeat=dim)],
                               dtype=np.int64)
        self.sp_xi = self.xi[self.sp_idx]                       # (nsp, dim)
        self.sp_w = np.prod(self.w[self.sp_idx], axis=1)        # tensor weights

        # flux points
        fp_dir, fp_side, fp_line = [], [], []
        face_idx = [t[::-1] for t in itertools.product(range(n), repeat=dim - 1)]
        for face in range(self.nfaces):
            k, side = face // 2, face % 2
            others = [a for a in range(dim) if a != k]
            for t in face_idx:
                full = [0] * dim
                for a, v in zip(others, t):
                    full[a] = v
                fp_dir.append(k)
                fp_side.append(side)
                fp_line.append(full)
        self.fp_dir = np.array(fp_dir)
        self.fp_side = np.array(fp_side)
        self.fp_sign = np.where(self.fp_side == 1, 1.0, -1.0)
        self.fp_face = np.repeat(np.arange(self.nfaces), self.nfpf)
        fp_line = np.array(fp_line, dtype=np.int64)
        self.fp_xi = self.xi[fp_line].astype(float)
        self.fp_xi[np.arange(self.nfp), self.fp_dir] = self.fp_sign
        # weight of the flux point in the face quadrature
        fw = np.ones(self.nfp)
        for f in range(self.nfp):
            for a in range(dim):
                if a != self.fp_dir[f]:
                    fw[f] *= self.w[fp_line[f, a]]
        self.fp_w = fw

        # lines: sp index at position m along the line of flux point f
        strides = n ** np.arange(dim)
        self.fp_line_sp = np.zeros((self.nfp, n), dtype=np.int64)
        for f in range(self.nfp):
            base = fp_line[f].copy()
            for m in range(n):
                base[self.fp_dir[f]] = m
                self.fp_line_sp[f, m] = int(np.dot(base, strides))

        # 1-D operators
        ends = basis.lagrange(self.xi, np.array([-1.0, 1.0]))    # (2, n)
        self.l_end = ends
        self.D1 = basis.lagrange_deriv(self.xi, self.xi)        # D1[i, m] = l_m'(xi_i)
        gL, gR, dgL, dgR = basis.correction_dg(p, self.xi)
        self.dgL, self.dgR = dgL, dgR

        nsp, nfp = self.nsp, self.nfp
        self.M0 = np.zeros((nfp, nsp))
        self.Cdiv = np.zeros((nsp, nfp))
        self.Cgrad = np.zeros((dim, nsp, nfp))
        for f in range(nfp):
            side = self.fp_side[f]
            k = self.fp_dir[f]
            for m in range(n):
                s = self.fp_line_sp[f, m]
                self.M0[f, s] = ends[side, m]
                if side == 1:
                    self.Cdiv[s, f] = dgR[m]
                    self.Cgrad[k, s, f] = dgR[m]
                else:
                    self.Cdiv[s, f] = -dgL[m]
                    self.Cgrad[k, s, f] = dgL[m]
        self.D = np.zeros((dim, nsp, nsp))
        for k in range(dim):
            for s in range(nsp):
                for m in range(n):
                    t = self.sp_idx[s].copy()
                    t[k] = m
                    s2 = int(np.dot(t, strides))
                    self.D[k, s, s2] = self.D1[self.sp_idx[s, k], m]

    def interp_matrix(self, xi_pts):
        """Tensor Lagrange basis of the solution points evaluated at
        reference points xi_pts (npts, dim): returns (npts, nsp)."""
        xi_pts = np.atleast_2d(xi_pts)
        out = np.ones((xi_pts.shape[0], self.nsp))
        for a in range(self.dim):
            La = basis.lagrange(self.xi, xi_pts[:, a])          # (npts, n)
            out *= La[:, self.sp_idx[:, a]]
        return out
