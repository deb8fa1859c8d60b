// Internal declarations shared by the host mesh code, the API and the kernel
// launchers of the FR library.  Not part of the public ABI (include/fr.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fr.h"

namespace fr {

constexpr int kMaxN = 5;        // p <= 4
constexpr int kMaxProbes = 1024;

// Tensor-product reference element on Gauss-Legendre points (Sec. 2.3, FR of
// Huynh with the DG-recovery correction).  Solution point s = i + n j (+ n^2 k);
// flux point f = face * n^(d-1) + l, faces -xi,+xi,-eta,+eta(,-zeta,+zeta),
// l running over the face's free directions, lower direction fastest.
struct RefElem {
    int dim = 0, p = 0, n = 0, nsp = 0, nfp = 0, nfpf = 0;
    double xi[kMaxN] = {}, w[kMaxN] = {};
    double lend[2][kMaxN] = {};          // l_m(-1), l_m(+1)
    double D1[kMaxN][kMaxN] = {};        // D1[i][m] = l_m'(xi_i)
    double dgL[kMaxN] = {}, dgR[kMaxN] = {};
    std::vector<double> sp_xi, fp_xi;    // reference coordinates
    std::vector<double> sp_w, fp_w;      // volume / face quadrature weights
    std::vector<int> fp_dir, fp_side;    // face-normal direction and side
};

void build_ref(RefElem &r, int dim, int p);
// sp index along the line of flux point f at position m
int ref_line_sp(const RefElem &r, int f, int m);
// tensor Lagrange basis of the solution points at reference point xi (dim)
void ref_interp(const RefElem &r, const double *xi, double *out);

}  // namespace fr

struct fr_mesh {
    int dim = 0, p = 0, q = 1;
    fr::RefElem ref;
    int64_t n_elem = 0;
    std::vector<double> nodes;     // n_elem * (q+1)^dim * dim geometry nodes
    std::vector<double> x_sp;      // n_elem * nsp * dim
    std::vector<double> S;         // n_elem * nsp * dim*dim, S[k][j] = J dxi_k/dx_j
    std::vector<double> J;         // n_elem * nsp
    std::vector<double> nrm;       // n_elem * nfp * dim, outward, scaled by |dS|
    std::vector<double> x_fp;      // n_elem * nfp * dim
    std::vector<int64_t> partner;  // n_elem * nfp, local e2 * nfp + f2 or -1
    std::vector<int32_t> bctag;    // n_elem * nfp, tag at boundary points, 0 else
};

namespace fr {
void set_error(const std::string &msg);
// Newton location of x in the mesh: element and reference coordinates.
bool mesh_locate(const fr_mesh &m, const double *x, int64_t *elem, double *xi);
}  // namespace fr
