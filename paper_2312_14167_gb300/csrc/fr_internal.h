// Internal declarations shared by the host mesh code, the API and the kernel
// launchers of the FR library.  Not part of the public ABI (include/fr.h).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "fr.h"

namespace fr {

constexpr int kMaxN = 5;        // p <= 4 (p = 0: one point, first-order finite volume)
constexpr int kMaxProbes = 1024;
// internal face tag of the flux points of a face joining an element of
// another degree (a mortar face); never passed in by a caller
constexpr int32_t kTagMortar = 64;

// One face joining elements of different degree, lower-degree side first.
// ``orient`` maps the higher side's face coordinates onto the lower side's:
// in 3-D (a, b) -> swap if bit 2, then a -> -a if bit 0, b -> -b if bit 1; in
// 2-D a -> -a if bit 0.
struct MortarLink {
    int part_lo = 0, part_hi = 0;   // parts (degrees) of the two sides
    int64_t e_lo = 0, e_hi = 0;     // element index within its part
    int f_lo = 0, f_hi = 0;         // face numbers
    int orient = 0;
};

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
// Mortar operators of a face: T [nfpf_hi][nfpf_lo], the lower face polynomial
// at the higher side's flux points; P [nfpf_lo][nfpf_hi], the L2 projection of
// the higher face polynomial onto the lower degree (Gauss quadrature of the
// higher side, exact for these degrees): P_ij = w_hi,j T_ji / w_lo,i.
void mortar_matrices(const RefElem &lo, const RefElem &hi, int orient, std::vector<double> &T,
                     std::vector<double> &P);
// sp index along the line of flux point f at position m
int ref_line_sp(const RefElem &r, int f, int m);
// tensor Lagrange basis of the solution points at reference point xi (dim)
void ref_interp(const RefElem &r, const double *xi, double *out);

}  // namespace fr

struct fr_mesh {
    int dim = 0, p = 0, q = 1;     // p = 0: the degree varies (see parts)
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
    // degree of each element and the number of solution points of the mesh
    std::vector<int32_t> elem_p;
    int64_t n_sp_total = 0;
    // A mesh with several degrees (fr_mesh_create_varp) keeps one uniform-degree
    // part per degree present, its elements in their relative order, faces to
    // other parts tagged kTagMortar, plus the list of those faces.  The fields
    // above then hold only dim, q, n_elem, nodes and x_sp (element order).  A
    // uniform mesh has no parts: it is its own single part.
    std::vector<std::unique_ptr<fr_mesh>> parts;
    std::vector<int32_t> part_of;  // part of each element
    std::vector<int64_t> local;    // index of each element within its part
    std::vector<fr::MortarLink> mortars;
};

namespace fr {
void set_error(const std::string &msg);
// Newton location of x in the mesh: element and reference coordinates.
bool mesh_locate(const fr_mesh &m, const double *x, int64_t *elem, double *xi);
}  // namespace fr
