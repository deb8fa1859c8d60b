// Host (FP64) mesh processing of the FR library: reference element, element
// maps, metric terms, normals and flux-point connectivity.
//
// Method: Flux Reconstruction (Sec. 2.3 of arXiv:2312.14167, Huynh's scheme)
// on tensor-product Gauss-Legendre points with the DG-recovery correction
// functions g_L = (-1)^(p+1)/2 (P_{p+1} - P_p), g_R = 1/2 (P_{p+1} + P_p).
// Geometry: the element map is the tensor Lagrange interpolant of equispaced
// geometry nodes; metric terms S[k][j] = J dxi_k/dx_j are the adjugate of the
// map Jacobian, evaluated analytically; the outward normal at a flux point is
// +-S[k][:] there.  All of this runs once per mesh in FP64; the FP32 solver
// casts the results.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>

#include "fr_internal.h"

namespace fr {

namespace {

// Legendre polynomial and derivative in long double (Bonnet recurrence).
void legendre_ld(int k, long double x, long double *P, long double *dP) {
    long double p0 = 1.0L, p1 = x, d0 = 0.0L, d1 = 1.0L;
    if (k == 0) { *P = 1.0L; *dP = 0.0L; return; }
    for (int n = 1; n < k; ++n) {
        long double p2 = ((2 * n + 1) * x * p1 - n * p0) / (n + 1);
        long double d2 = d0 + (2 * n + 1) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    *P = p1; *dP = d1;
}

double lagrange_1d(const double *nodes, int n, int j, double x) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != j) v *= (x - nodes[m]) / (nodes[j] - nodes[m]);
    return v;
}

double lagrange_1d_deriv(const double *nodes, int n, int j, double x) {
    double denom = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != j) denom *= nodes[j] - nodes[m];
    double s = 0.0;
    for (int r = 0; r < n; ++r) {
        if (r == j) continue;
        double t = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != j && m != r) t *= x - nodes[m];
        s += t;
    }
    return s / denom;
}

}  // namespace

void build_ref(RefElem &r, int dim, int p) {
    const int n = p + 1;
    r.dim = dim; r.p = p; r.n = n;
    r.nsp = (dim == 2) ? n * n : n * n * n;
    r.nfpf = (dim == 2) ? n : n * n;
    r.nfp = 2 * dim * r.nfpf;
    // Gauss-Legendre nodes: Newton in long double from Chebyshev-like guesses
    for (int i = 0; i < n; ++i) {
        long double x = -cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (n + 0.5L));
        for (int it = 0; it < 200; ++it) {
            long double P, dP;
            legendre_ld(n, x, &P, &dP);
            long double dx = P / dP;
            x -= dx;
            if (fabsl(dx) < 1e-19L) break;
        }
        long double P, dP;
        legendre_ld(n, x, &P, &dP);
        r.xi[i] = (double)x;
        r.w[i] = (double)(2.0L / ((1.0L - x * x) * dP * dP));
    }
    for (int m = 0; m < n; ++m) {
        r.lend[0][m] = lagrange_1d(r.xi, n, m, -1.0);
        r.lend[1][m] = lagrange_1d(r.xi, n, m, 1.0);
        for (int i = 0; i < n; ++i) r.D1[i][m] = lagrange_1d_deriv(r.xi, n, m, r.xi[i]);
    }
    const long double sgn = (p % 2 == 0) ? -0.5L : 0.5L;   // (-1)^(p+1) / 2
    for (int i = 0; i < n; ++i) {
        long double P1, dP1, P0, dP0;
        legendre_ld(p + 1, r.xi[i], &P1, &dP1);
        legendre_ld(p, r.xi[i], &P0, &dP0);
        r.dgL[i] = (double)(sgn * (dP1 - dP0));
        r.dgR[i] = (double)(0.5L * (dP1 + dP0));
    }
    r.sp_xi.assign((size_t)r.nsp * dim, 0.0);
    r.sp_w.assign(r.nsp, 1.0);
    for (int s = 0; s < r.nsp; ++s) {
        int t = s;
        for (int a = 0; a < dim; ++a) {
            int ia = t % n; t /= n;
            r.sp_xi[(size_t)s * dim + a] = r.xi[ia];
            r.sp_w[s] *= r.w[ia];
        }
    }
    r.fp_xi.assign((size_t)r.nfp * dim, 0.0);
    r.fp_w.assign(r.nfp, 1.0);
    r.fp_dir.assign(r.nfp, 0);
    r.fp_side.assign(r.nfp, 0);
    for (int f = 0; f < r.nfp; ++f) {
        const int face = f / r.nfpf, l = f % r.nfpf, k = face / 2, side = face % 2;
        r.fp_dir[f] = k; r.fp_side[f] = side;
        int t = l;
        for (int a = 0; a < dim; ++a) {
            if (a == k) { r.fp_xi[(size_t)f * dim + a] = side ? 1.0 : -1.0; continue; }
            int ia = t % n; t /= n;
            r.fp_xi[(size_t)f * dim + a] = r.xi[ia];
            r.fp_w[f] *= r.w[ia];
        }
    }
}

int ref_line_sp(const RefElem &r, int f, int m) {
    const int n = r.n, face = f / r.nfpf, k = face / 2;
    int l = f % r.nfpf, idx[3] = {0, 0, 0};
    for (int a = 0; a < r.dim; ++a) {
        if (a == k) { idx[a] = m; continue; }
        idx[a] = l % n; l /= n;
    }
    return idx[0] + n * idx[1] + n * n * idx[2];
}

void ref_interp(const RefElem &r, const double *xi, double *out) {
    const int n = r.n;
    double L[3][kMaxN];
    for (int a = 0; a < r.dim; ++a)
        for (int m = 0; m < n; ++m) L[a][m] = lagrange_1d(r.xi, n, m, xi[a]);
    for (int s = 0; s < r.nsp; ++s) {
        int t = s;
        double v = 1.0;
        for (int a = 0; a < r.dim; ++a) { v *= L[a][t % n]; t /= n; }
        out[s] = v;
    }
}

// --------------------------------------------------------------------------
// element map
// --------------------------------------------------------------------------
namespace {

struct MapEval {
    int dim, q, nn;
    std::vector<double> eq;
    explicit MapEval(int dim_, int q_) : dim(dim_), q(q_) {
        nn = 1;
        for (int a = 0; a < dim; ++a) nn *= (q + 1);
        eq.resize(q + 1);
        for (int i = 0; i <= q; ++i) eq[i] = -1.0 + 2.0 * i / q;
    }
    // x (dim) and A[j][k] = dx_j/dxi_k at xi, from the element's nodes.  The
    // sums run over offsets from node 0 (the shape functions sum to one and
    // their derivatives to zero), so rounding scales with the element size.
    void eval(const double *nodes, const double *xi, double *x, double A[3][3]) const {
        double L[3][8], dL[3][8];
        for (int a = 0; a < dim; ++a)
            for (int m = 0; m <= q; ++m) {
                L[a][m] = lagrange_1d(eq.data(), q + 1, m, xi[a]);
                dL[a][m] = lagrange_1d_deriv(eq.data(), q + 1, m, xi[a]);
            }
        for (int j = 0; j < dim; ++j) {
            x[j] = 0.0;
            for (int k = 0; k < dim; ++k) A[j][k] = 0.0;
        }
        for (int a = 0; a < nn; ++a) {
            int idx[3] = {0, 0, 0}, t = a;
            for (int d = 0; d < dim; ++d) { idx[d] = t % (q + 1); t /= (q + 1); }
            double N = 1.0, dN[3];
            for (int d = 0; d < dim; ++d) N *= L[d][idx[d]];
            for (int k = 0; k < dim; ++k) {
                dN[k] = 1.0;
                for (int d = 0; d < dim; ++d) dN[k] *= (d == k) ? dL[d][idx[d]] : L[d][idx[d]];
            }
            for (int j = 0; j < dim; ++j) {
                const double X = nodes[(size_t)a * dim + j] - nodes[j];
                x[j] += N * X;
                for (int k = 0; k < dim; ++k) A[j][k] += dN[k] * X;
            }
        }
        for (int j = 0; j < dim; ++j) x[j] += nodes[j];
    }
};

// Shape functions of the map and their derivatives tabulated at a fixed set
// of reference points (the same for every element).
struct MapTable {
    int dim = 0, nn = 0, npts = 0;
    std::vector<double> N, dN;   // N[p*nn + a], dN[(p*nn + a)*3 + k]
    MapTable(const MapEval &me, const std::vector<double> &xi, int npts_) : dim(me.dim), nn(me.nn), npts(npts_) {
        N.assign((size_t)npts * nn, 0.0);
        dN.assign((size_t)npts * nn * 3, 0.0);
        // evaluate with unit node vectors: x = sum_a N_a X_a picks N_a
        std::vector<double> unit((size_t)nn * dim, 0.0);
        for (int pt = 0; pt < npts; ++pt) {
            double L[3][8], dL[3][8];
            for (int a = 0; a < dim; ++a)
                for (int m = 0; m <= me.q; ++m) {
                    L[a][m] = lagrange_1d(me.eq.data(), me.q + 1, m, xi[(size_t)pt * dim + a]);
                    dL[a][m] = lagrange_1d_deriv(me.eq.data(), me.q + 1, m, xi[(size_t)pt * dim + a]);
                }
            for (int a = 0; a < nn; ++a) {
                int idx[3] = {0, 0, 0}, t = a;
                for (int d = 0; d < dim; ++d) { idx[d] = t % (me.q + 1); t /= (me.q + 1); }
                double n = 1.0;
                for (int d = 0; d < dim; ++d) n *= L[d][idx[d]];
                N[(size_t)pt * nn + a] = n;
                for (int k = 0; k < dim; ++k) {
                    double v = 1.0;
                    for (int d = 0; d < dim; ++d) v *= (d == k) ? dL[d][idx[d]] : L[d][idx[d]];
                    dN[((size_t)pt * nn + a) * 3 + k] = v;
                }
            }
        }
    }
    // same arithmetic as MapEval::eval (offsets from node 0), tabulated
    void eval(const double *nodes, int pt, double *x, double A[3][3]) const {
        for (int j = 0; j < dim; ++j) {
            x[j] = 0.0;
            for (int k = 0; k < dim; ++k) A[j][k] = 0.0;
        }
        const double *n = &N[(size_t)pt * nn];
        const double *dn = &dN[(size_t)pt * nn * 3];
        for (int a = 0; a < nn; ++a)
            for (int j = 0; j < dim; ++j) {
                const double X = nodes[(size_t)a * dim + j] - nodes[j];
                x[j] += n[a] * X;
                for (int k = 0; k < dim; ++k) A[j][k] += dn[a * 3 + k] * X;
            }
        for (int j = 0; j < dim; ++j) x[j] += nodes[j];
    }
};

// S[k][j] = J dxi_k / dx_j (adjugate of A), returns J
double adjugate(int dim, const double A[3][3], double S[3][3]) {
    if (dim == 2) {
        S[0][0] = A[1][1];  S[0][1] = -A[0][1];
        S[1][0] = -A[1][0]; S[1][1] = A[0][0];
        return A[0][0] * A[1][1] - A[0][1] * A[1][0];
    }
    for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        // row k = (dx/dxi_k1) x (dx/dxi_k2)
        S[k][0] = A[1][k1] * A[2][k2] - A[2][k1] * A[1][k2];
        S[k][1] = A[2][k1] * A[0][k2] - A[0][k1] * A[2][k2];
        S[k][2] = A[0][k1] * A[1][k2] - A[1][k1] * A[0][k2];
    }
    return A[0][0] * S[0][0] + A[1][0] * S[0][1] + A[2][0] * S[0][2];
}

const int kQuadFaces[4][2] = {{0, 2}, {1, 3}, {0, 1}, {2, 3}};
const int kHexFaces[6][4] = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5},
                             {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};

struct Key4 {
    std::array<int64_t, 4> v;
    bool operator==(const Key4 &o) const { return v == o.v; }
};
struct Key4Hash {
    size_t operator()(const Key4 &k) const {
        uint64_t h = 1469598103934665603ull;
        for (int64_t x : k.v) { h ^= (uint64_t)x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2); }
        return (size_t)h;
    }
};

}  // namespace

bool mesh_locate(const fr_mesh &m, const double *x, int64_t *elem, double *xi) {
    MapEval me(m.dim, m.q);
    const int d = m.dim;
    for (int64_t e = 0; e < m.n_elem; ++e) {
        const double *nd = &m.nodes[(size_t)e * me.nn * d];
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int a = 0; a < me.nn; ++a)
            for (int j = 0; j < d; ++j) {
                lo[j] = std::min(lo[j], nd[a * d + j]);
                hi[j] = std::max(hi[j], nd[a * d + j]);
            }
        double span = 0;
        for (int j = 0; j < d; ++j) span = std::max(span, hi[j] - lo[j]);
        bool inside = true;
        for (int j = 0; j < d; ++j)
            if (x[j] < lo[j] - 1e-9 * span || x[j] > hi[j] + 1e-9 * span) inside = false;
        if (!inside) continue;
        double z[3] = {0, 0, 0};
        bool ok = true;
        for (int it = 0; it < 60; ++it) {
            double xx[3], A[3][3], S[3][3];
            me.eval(nd, z, xx, A);
            const double J = adjugate(d, A, S);
            if (J == 0.0) { ok = false; break; }
            double r[3] = {x[0] - xx[0], x[1] - xx[1], d == 3 ? x[2] - xx[2] : 0.0};
            double dz[3] = {0, 0, 0}, mx = 0;
            // A^{-1} = S / J (S is the adjugate)
            for (int k = 0; k < d; ++k) {
                for (int j = 0; j < d; ++j) dz[k] += S[k][j] * r[j] / J;
                z[k] += dz[k];
                mx = std::max(mx, std::fabs(dz[k]));
            }
            if (std::fabs(z[0]) > 3 || std::fabs(z[1]) > 3 || (d == 3 && std::fabs(z[2]) > 3)) { ok = false; break; }
            if (mx < 1e-14) break;
        }
        if (!ok) continue;
        bool in = true;
        for (int k = 0; k < d; ++k) in = in && std::fabs(z[k]) <= 1.0 + 1e-10;
        if (!in) continue;
        *elem = e;
        for (int k = 0; k < d; ++k) xi[k] = std::max(-1.0, std::min(1.0, z[k]));
        return true;
    }
    return false;
}

}  // namespace fr

using fr::RefElem;

namespace fr {
namespace {

// One connected face seen from one side: corners of (e, fc) + sh lie on those
// of (e2, fc2).  Global element indices.
struct Pair { int64_t e; int fc; int64_t e2; int fc2; double sh[3]; };

struct MeshInput {
    int dim;
    int64_t n_vert, n_elem;
    const double *xyz;
    const int64_t *elem_vert;
    const int32_t *face_tag;
    int n_shift;
    const double *periodic_shift;
    int64_t corner(int64_t e, int fc, int c) const {
        const int nc = 1 << dim;
        return dim == 2 ? elem_vert[e * nc + kQuadFaces[fc][c]] : elem_vert[e * nc + kHexFaces[fc][c]];
    }
    int ncf() const { return dim == 2 ? 2 : 4; }
};

// Interior faces share their corner vertices; periodic faces are matched by
// corner coordinates (rounded on a fine lattice) after adding or subtracting
// one of the periodic shifts.
fr_status find_face_pairs(const MeshInput &in, std::vector<Pair> &pairs) {
    const int dim = in.dim, ncf = in.ncf();
    std::unordered_map<Key4, std::vector<std::pair<int64_t, int>>, Key4Hash> by_ids;
    by_ids.reserve((size_t)in.n_elem * dim * 2);
    for (int64_t e = 0; e < in.n_elem; ++e)
        for (int fc = 0; fc < 2 * dim; ++fc) {
            const int32_t tg = in.face_tag[e * 2 * dim + fc];
            if (tg < 0 || tg > 5) {
                set_error("fr_mesh_create: unknown face tag");
                return FR_ERR_INVALID_ARG;
            }
            if (tg != FR_TAG_INTERIOR) continue;
            Key4 k{{-1, -1, -1, -1}};
            for (int c = 0; c < ncf; ++c) k.v[c] = in.corner(e, fc, c);
            std::sort(k.v.begin(), k.v.begin() + ncf);
            by_ids[k].push_back({e, fc});
        }
    for (auto &kv : by_ids) {
        if (kv.second.size() != 2) {
            set_error("fr_mesh_create: interior face without exactly one partner");
            return FR_ERR_MESH;
        }
        auto a = kv.second[0], b = kv.second[1];
        pairs.push_back({a.first, a.second, b.first, b.second, {0, 0, 0}});
        pairs.push_back({b.first, b.second, a.first, a.second, {0, 0, 0}});
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t v = 0; v < in.n_vert; ++v)
        for (int j = 0; j < dim; ++j) {
            lo[j] = std::min(lo[j], in.xyz[v * dim + j]);
            hi[j] = std::max(hi[j], in.xyz[v * dim + j]);
        }
    double span = 0;
    for (int j = 0; j < dim; ++j) span = std::max(span, hi[j] - lo[j]);
    const double scale = 1e6 / std::max(span, 1e-300);
    using CKey = std::vector<int64_t>;
    std::map<CKey, std::pair<int64_t, int>> table;
    auto ckey = [&](int64_t e, int fc, const double *sh) {
        std::vector<std::array<int64_t, 3>> pts(ncf);
        for (int c = 0; c < ncf; ++c) {
            const int64_t v = in.corner(e, fc, c);
            for (int j = 0; j < 3; ++j)
                pts[c][j] = j < dim ? (int64_t)std::llround((in.xyz[v * dim + j] + (sh ? sh[j] : 0.0)) * scale) : 0;
        }
        std::sort(pts.begin(), pts.end());
        CKey k;
        for (auto &pt : pts) k.insert(k.end(), pt.begin(), pt.end());
        return k;
    };
    std::vector<std::pair<int64_t, int>> per;
    for (int64_t e = 0; e < in.n_elem; ++e)
        for (int fc = 0; fc < 2 * dim; ++fc)
            if (in.face_tag[e * 2 * dim + fc] == FR_TAG_PERIODIC) {
                per.push_back({e, fc});
                table[ckey(e, fc, nullptr)] = {e, fc};
            }
    for (auto &pf : per) {
        bool found = false;
        for (int s = 0; s < in.n_shift && !found; ++s)
            for (int sg = 1; sg >= -1 && !found; sg -= 2) {
                double sh[3] = {0, 0, 0};
                for (int j = 0; j < dim; ++j) sh[j] = sg * in.periodic_shift[s * dim + j];
                auto it = table.find(ckey(pf.first, pf.second, sh));
                if (it != table.end() && it->second != pf) {
                    pairs.push_back({pf.first, pf.second, it->second.first, it->second.second,
                                     {sh[0], sh[1], sh[2]}});
                    found = true;
                }
            }
        if (!found) {
            set_error("fr_mesh_create: periodic face without partner");
            return FR_ERR_MESH;
        }
    }
    return FR_OK;
}

// Metric terms, normals and point coordinates of a uniform-degree part whose
// ref, q, n_elem and nodes are set.
fr_status build_geometry(fr_mesh *m) {
    const RefElem &r = m->ref;
    const int dim = m->dim, nsp = r.nsp, nfp = r.nfp;
    const int64_t n_elem = m->n_elem;
    MapEval me(dim, m->q);
    m->x_sp.resize((size_t)n_elem * nsp * dim);
    m->S.resize((size_t)n_elem * nsp * dim * dim);
    m->J.resize((size_t)n_elem * nsp);
    m->nrm.resize((size_t)n_elem * nfp * dim);
    m->x_fp.resize((size_t)n_elem * nfp * dim);
    m->partner.assign((size_t)n_elem * nfp, -1);
    m->bctag.assign((size_t)n_elem * nfp, 0);
    const MapTable tsp(me, r.sp_xi, nsp), tfp(me, r.fp_xi, nfp);
    int64_t bad_elem = -1;
    // elements are independent: one host thread per chunk of elements
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_elem; ++e) {
        const double *nd = &m->nodes[(size_t)e * me.nn * dim];
        for (int s = 0; s < nsp; ++s) {
            double x[3], A[3][3], S[3][3];
            tsp.eval(nd, s, x, A);
            const double J = adjugate(dim, A, S);
            if (!(J > 0.0)) {
#pragma omp critical
                {
                    if (bad_elem < 0 || e < bad_elem) bad_elem = e;
                }
            }
            m->J[(size_t)e * nsp + s] = J;
            for (int j = 0; j < dim; ++j) m->x_sp[((size_t)e * nsp + s) * dim + j] = x[j];
            for (int k = 0; k < dim; ++k)
                for (int j = 0; j < dim; ++j)
                    m->S[(((size_t)e * nsp + s) * dim + k) * dim + j] = S[k][j];
        }
        for (int f = 0; f < nfp; ++f) {
            double x[3], A[3][3], S[3][3];
            tfp.eval(nd, f, x, A);
            adjugate(dim, A, S);
            const int k = r.fp_dir[f];
            const double sg = r.fp_side[f] ? 1.0 : -1.0;
            for (int j = 0; j < dim; ++j) {
                m->nrm[((size_t)e * nfp + f) * dim + j] = sg * S[k][j];
                m->x_fp[((size_t)e * nfp + f) * dim + j] = x[j];
            }
        }
    }
    if (bad_elem >= 0) {
        set_error("fr_mesh_create: non-positive Jacobian in element " + std::to_string(bad_elem));
        return FR_ERR_MESH;
    }
    return FR_OK;
}

double face_hmin(const MeshInput &in, int64_t e, int fc) {
    double hmin = 1e300;
    const int ncf = in.ncf();
    for (int i = 0; i < ncf; ++i)
        for (int j = i + 1; j < ncf; ++j) {
            double q2 = 0;
            for (int c = 0; c < in.dim; ++c) {
                const double dd = in.xyz[in.corner(e, fc, i) * in.dim + c] - in.xyz[in.corner(e, fc, j) * in.dim + c];
                q2 += dd * dd;
            }
            hmin = std::min(hmin, std::sqrt(q2));
        }
    return hmin;
}

// Pair the flux points of two connected faces of one part by physical
// position.  A face's points form an n x n (3-D) or n (2-D) tensor grid, so
// the partner's numbering is one of the 8 (3-D) or 2 (2-D) orientations of
// that grid: choose it on three reference points, then check every point.
fr_status pair_points(fr_mesh *m, int64_t e, int fc, int64_t e2, int fc2, const double *sh, double hmin) {
    const RefElem &r = m->ref;
    const int dim = m->dim, nfp = r.nfp, nfpf = r.nfpf, nn1 = r.n;
    auto orient = [&](int o, int a) -> int {
        if (dim == 2) return o ? nn1 - 1 - a : a;
        int i = a % nn1, j = a / nn1;
        if (o & 4) std::swap(i, j);
        if (o & 1) i = nn1 - 1 - i;
        if (o & 2) j = nn1 - 1 - j;
        return i + nn1 * j;
    };
    const int n_orient = dim == 2 ? 2 : 8;
    const int refs[3] = {0, nfpf - 1, dim == 2 ? nfpf / 2 : nn1 - 1};
    const double *xa = &m->x_fp[((size_t)e * nfp + fc * nfpf) * dim];
    const double *xb = &m->x_fp[((size_t)e2 * nfp + fc2 * nfpf) * dim];
    auto d2 = [&](int a, int b) {
        double t = 0;
        for (int c = 0; c < dim; ++c) {
            const double dd = xa[a * dim + c] + sh[c] - xb[b * dim + c];
            t += dd * dd;
        }
        return t;
    };
    int best = 0;
    double bd = 1e300;
    for (int o = 0; o < n_orient; ++o) {
        double t = 0;
        for (int rr = 0; rr < 3; ++rr) t += d2(refs[rr], orient(o, refs[rr]));
        if (t < bd) { bd = t; best = o; }
    }
    for (int a = 0; a < nfpf; ++a) {
        const int b = orient(best, a);
        if (std::sqrt(d2(a, b)) > 1e-6 * hmin) {
            set_error("fr_mesh_create: flux points of a connected face do not coincide");
            return FR_ERR_MESH;
        }
        m->partner[(size_t)e * nfp + fc * nfpf + a] = e2 * nfp + fc2 * nfpf + b;
    }
    return FR_OK;
}

// Physical position of face coordinates c (d-1 values in [-1, 1]) on face fc
// of an element with nodes nd.
void face_point(const MapEval &me, const double *nd, int fc, const double *c, double *x) {
    const int dim = me.dim, k = fc / 2;
    double xi[3] = {0, 0, 0};
    int t = 0;
    for (int a = 0; a < dim; ++a) xi[a] = (a == k) ? ((fc & 1) ? 1.0 : -1.0) : c[t++];
    double A[3][3];
    me.eval(nd, xi, x, A);
}

void apply_orient(int dim, int o, const double *c, double *out) {
    if (dim == 2) { out[0] = (o & 1) ? -c[0] : c[0]; return; }
    double a = c[0], b = c[1];
    if (o & 4) std::swap(a, b);
    if (o & 1) a = -a;
    if (o & 2) b = -b;
    out[0] = a; out[1] = b;
}

// Orientation mapping the higher face's coordinates onto the lower face's,
// from the corners' physical positions (lower + sh lies on higher).
fr_status mortar_orient(const MeshInput &in, const MapEval &me, const std::vector<double> &nodes,
                        const Pair &lo_hi, double hmin, int *orient) {
    const int dim = in.dim, ncorner = dim == 2 ? 2 : 4, n_orient = dim == 2 ? 2 : 8;
    const double *nl = &nodes[(size_t)lo_hi.e * me.nn * dim];
    const double *nh = &nodes[(size_t)lo_hi.e2 * me.nn * dim];
    int best = -1;
    double bd = 1e300;
    for (int o = 0; o < n_orient; ++o) {
        double worst = 0;
        for (int c = 0; c < ncorner; ++c) {
            const double ch[2] = {(c & 1) ? 1.0 : -1.0, (c & 2) ? 1.0 : -1.0};
            double cl[2], xh[3], xl[3];
            apply_orient(dim, o, ch, cl);
            face_point(me, nh, lo_hi.fc2, ch, xh);
            face_point(me, nl, lo_hi.fc, cl, xl);
            double t = 0;
            for (int j = 0; j < dim; ++j) {
                const double dd = xl[j] + lo_hi.sh[j] - xh[j];
                t += dd * dd;
            }
            worst = std::max(worst, t);
        }
        if (worst < bd) { bd = worst; best = o; }
    }
    if (best < 0 || std::sqrt(bd) > 1e-6 * hmin) {
        set_error("fr_mesh_create: corners of a face joining two degrees do not coincide");
        return FR_ERR_MESH;
    }
    *orient = best;
    return FR_OK;
}

fr_status mesh_create_impl(fr_mesh **out, int dim, int p_uniform, const int32_t *elem_p, int64_t n_vert,
                           const double *xyz, int64_t n_elem, const int64_t *elem_vert, int geo_order,
                           const double *geo_nodes, const int32_t *face_tag, int n_shift,
                           const double *periodic_shift) {
    if (!out || !xyz || !elem_vert || !face_tag || n_elem <= 0 || n_vert <= 0 ||
        (dim != 2 && dim != 3) || geo_order < 1 || geo_order > 7 ||
        (n_shift > 0 && !periodic_shift) || n_shift < 0) {
        set_error("fr_mesh_create: invalid argument");
        return FR_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::vector<int32_t> degree((size_t)n_elem, p_uniform);
    if (elem_p) std::copy(elem_p, elem_p + n_elem, degree.begin());
    bool present[kMaxN] = {};
    for (int64_t e = 0; e < n_elem; ++e) {
        if (degree[e] < 0 || degree[e] > 4) {
            set_error("fr_mesh_create: polynomial degree must be 0..4");
            return FR_ERR_UNSUPPORTED;
        }
        present[degree[e]] = true;
    }
    const int nc = 1 << dim;
    for (int64_t i = 0; i < n_elem * nc; ++i)
        if (elem_vert[i] < 0 || elem_vert[i] >= n_vert) {
            set_error("fr_mesh_create: vertex index out of range");
            return FR_ERR_INVALID_ARG;
        }
    const MeshInput in{dim, n_vert, n_elem, xyz, elem_vert, face_tag, n_shift, periodic_shift};
    // geometry nodes of every element
    const int q = geo_nodes ? geo_order : 1;
    MapEval me(dim, q);
    std::vector<double> nodes((size_t)n_elem * me.nn * dim);
    if (geo_nodes) {
        std::memcpy(nodes.data(), geo_nodes, nodes.size() * sizeof(double));
    } else {
        for (int64_t e = 0; e < n_elem; ++e)
            for (int c = 0; c < nc; ++c)
                for (int j = 0; j < dim; ++j)
                    nodes[((size_t)e * nc + c) * dim + j] = xyz[elem_vert[e * nc + c] * dim + j];
    }
    std::vector<Pair> pairs;
    fr_status st = find_face_pairs(in, pairs);
    if (st != FR_OK) return st;

    // one part per degree present, elements in their relative order
    int part_of_degree[kMaxN] = {-1, -1, -1, -1, -1}, n_parts = 0;
    for (int d = 0; d < kMaxN; ++d)
        if (present[d]) part_of_degree[d] = n_parts++;
    std::vector<int32_t> part_of((size_t)n_elem);
    std::vector<int64_t> local((size_t)n_elem);
    std::vector<int64_t> count(n_parts, 0);
    for (int64_t e = 0; e < n_elem; ++e) {
        part_of[e] = part_of_degree[degree[e]];
        local[e] = count[part_of[e]]++;
    }
    std::vector<std::unique_ptr<fr_mesh>> parts(n_parts);
    for (int d = 0; d < kMaxN; ++d) {
        const int pi = part_of_degree[d];
        if (pi < 0) continue;
        auto pm = std::make_unique<fr_mesh>();
        pm->dim = dim; pm->p = d; pm->q = q; pm->n_elem = count[pi];
        build_ref(pm->ref, dim, d);
        if (n_parts == 1) {
            pm->nodes = std::move(nodes);
        } else {
            pm->nodes.resize((size_t)count[pi] * me.nn * dim);
            for (int64_t e = 0; e < n_elem; ++e)
                if (part_of[e] == pi)
                    std::memcpy(&pm->nodes[(size_t)local[e] * me.nn * dim], &nodes[(size_t)e * me.nn * dim],
                                (size_t)me.nn * dim * sizeof(double));
        }
        st = build_geometry(pm.get());
        if (st != FR_OK) return st;
        pm->elem_p.assign((size_t)count[pi], d);
        pm->n_sp_total = count[pi] * pm->ref.nsp;
        parts[pi] = std::move(pm);
    }
    const std::vector<double> &all_nodes = n_parts == 1 ? parts[0]->nodes : nodes;

    std::vector<MortarLink> mortars;
    for (const Pair &pr : pairs) {
        const int pa = part_of[pr.e], pb = part_of[pr.e2];
        fr_mesh *ma = parts[pa].get();
        if (pa == pb) {
            st = pair_points(ma, local[pr.e], pr.fc, local[pr.e2], pr.fc2, pr.sh, face_hmin(in, pr.e, pr.fc));
            if (st != FR_OK) return st;
            continue;
        }
        for (int a = 0; a < ma->ref.nfpf; ++a)
            ma->bctag[(size_t)local[pr.e] * ma->ref.nfp + pr.fc * ma->ref.nfpf + a] = kTagMortar;
        if (degree[pr.e] < degree[pr.e2]) {
            MortarLink L;
            L.part_lo = pa; L.part_hi = pb;
            L.e_lo = local[pr.e]; L.e_hi = local[pr.e2];
            L.f_lo = pr.fc; L.f_hi = pr.fc2;
            st = mortar_orient(in, me, all_nodes, pr, face_hmin(in, pr.e, pr.fc), &L.orient);
            if (st != FR_OK) return st;
            mortars.push_back(L);
        }
    }
    for (int64_t e = 0; e < n_elem; ++e) {
        fr_mesh *pm = parts[part_of[e]].get();
        const int nfp = pm->ref.nfp, nfpf = pm->ref.nfpf;
        for (int fc = 0; fc < 2 * dim; ++fc) {
            const int32_t tg = face_tag[e * 2 * dim + fc];
            for (int a = 0; a < nfpf; ++a) {
                const size_t i = (size_t)local[e] * nfp + fc * nfpf + a;
                if (tg >= FR_TAG_WALL) {
                    pm->bctag[i] = tg;
                } else if (pm->partner[i] < 0 && pm->bctag[i] != kTagMortar) {
                    set_error("fr_mesh_create: face left unconnected");
                    return FR_ERR_MESH;
                }
            }
        }
    }
    if (n_parts == 1) {
        *out = parts[0].release();
        return FR_OK;
    }
    auto m = std::make_unique<fr_mesh>();
    m->dim = dim; m->p = 0; m->q = q; m->n_elem = n_elem;
    m->nodes = std::move(nodes);
    m->elem_p = degree;
    m->part_of = std::move(part_of);
    m->local = std::move(local);
    m->mortars = std::move(mortars);
    for (int64_t e = 0; e < n_elem; ++e) {
        const fr_mesh *pm = parts[m->part_of[e]].get();
        const size_t n = (size_t)pm->ref.nsp * dim;
        m->x_sp.insert(m->x_sp.end(), pm->x_sp.begin() + m->local[e] * n, pm->x_sp.begin() + (m->local[e] + 1) * n);
        m->n_sp_total += pm->ref.nsp;
    }
    m->parts = std::move(parts);
    *out = m.release();
    return FR_OK;
}

double lagrange_at(const RefElem &r, int j, double x) { return lagrange_1d(r.xi, r.n, j, x); }

}  // namespace

void mortar_matrices(const RefElem &lo, const RefElem &hi, int orient, std::vector<double> &T,
                     std::vector<double> &P) {
    const int dim = lo.dim, nl = lo.nfpf, nh = hi.nfpf;
    T.assign((size_t)nh * nl, 0.0);
    P.assign((size_t)nl * nh, 0.0);
    auto face_w = [&](const RefElem &r, int i) { return dim == 2 ? r.w[i] : r.w[i % r.n] * r.w[i / r.n]; };
    for (int j = 0; j < nh; ++j) {
        const double ch[2] = {hi.xi[j % hi.n], dim == 3 ? hi.xi[j / hi.n] : 0.0};
        double cl[2] = {0, 0};
        apply_orient(dim, orient, ch, cl);
        for (int i = 0; i < nl; ++i) {
            double v = lagrange_at(lo, i % lo.n, cl[0]);
            if (dim == 3) v *= lagrange_at(lo, i / lo.n, cl[1]);
            T[(size_t)j * nl + i] = v;
        }
    }
    for (int i = 0; i < nl; ++i)
        for (int j = 0; j < nh; ++j)
            P[(size_t)i * nh + j] = face_w(hi, j) * T[(size_t)j * nl + i] / face_w(lo, i);
}

}  // namespace fr

extern "C" fr_status fr_mesh_create(fr_mesh **out, int dim, int p, int64_t n_vert,
                                    const double *xyz, int64_t n_elem, const int64_t *elem_vert,
                                    int geo_order, const double *geo_nodes,
                                    const int32_t *face_tag, int n_shift,
                                    const double *periodic_shift) {
    if (out && (p < 0 || p > 4)) {
        *out = nullptr;
        fr::set_error("fr_mesh_create: polynomial degree must be 0..4");
        return FR_ERR_UNSUPPORTED;
    }
    return fr::mesh_create_impl(out, dim, p, nullptr, n_vert, xyz, n_elem, elem_vert, geo_order, geo_nodes,
                                face_tag, n_shift, periodic_shift);
}

extern "C" fr_status fr_mesh_create_varp(fr_mesh **out, int dim, const int32_t *elem_p, int64_t n_vert,
                                         const double *xyz, int64_t n_elem, const int64_t *elem_vert,
                                         int geo_order, const double *geo_nodes,
                                         const int32_t *face_tag, int n_shift,
                                         const double *periodic_shift) {
    if (!elem_p) {
        if (out) *out = nullptr;
        fr::set_error("fr_mesh_create_varp: null degree array");
        return FR_ERR_INVALID_ARG;
    }
    return fr::mesh_create_impl(out, dim, 0, elem_p, n_vert, xyz, n_elem, elem_vert, geo_order, geo_nodes,
                                face_tag, n_shift, periodic_shift);
}

extern "C" void fr_mesh_destroy(fr_mesh *mesh) { delete mesh; }

extern "C" fr_status fr_mesh_info(const fr_mesh *m, int64_t *n_elem, int *nsp, int *nfp) {
    if (!m) { fr::set_error("fr_mesh_info: null mesh"); return FR_ERR_INVALID_ARG; }
    const bool uniform = m->parts.empty();
    if (n_elem) *n_elem = m->n_elem;
    if (nsp) *nsp = uniform ? m->ref.nsp : 0;
    if (nfp) *nfp = uniform ? m->ref.nfp : 0;
    return FR_OK;
}

extern "C" fr_status fr_mesh_degrees(const fr_mesh *m, int32_t *elem_p, int64_t *n_sol_points) {
    if (!m) { fr::set_error("fr_mesh_degrees: null mesh"); return FR_ERR_INVALID_ARG; }
    if (elem_p) std::copy(m->elem_p.begin(), m->elem_p.end(), elem_p);
    if (n_sol_points) *n_sol_points = m->n_sp_total;
    return FR_OK;
}

extern "C" fr_status fr_mesh_sol_coords(const fr_mesh *m, double *xyz) {
    if (!m || !xyz) { fr::set_error("fr_mesh_sol_coords: null argument"); return FR_ERR_INVALID_ARG; }
    std::memcpy(xyz, m->x_sp.data(), m->x_sp.size() * sizeof(double));
    return FR_OK;
}
