// C ABI of the FR library (include/fr.h): batch solver object, workspace
// carving, CUDA-graph replay of the RK step, probes, OASPL and the FP64
// reductions.  Kernels live in fr_kernels.cuh, instantiated per dimension and
// precision in fr_k{2,3}_{f32,f64}.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "fr_internal.h"
#include "fr_kernels.cuh"

namespace frk {
cudaError_t launch_2_f32(int N, int kind, bool visc, const KArgs<float> &a, int grid, cudaStream_t s);
cudaError_t launch_2_f64(int N, int kind, bool visc, const KArgs<double> &a, int grid, cudaStream_t s);
cudaError_t launch_3_f32(int N, int kind, bool visc, const KArgs<float> &a, int grid, cudaStream_t s);
cudaError_t launch_3_f64(int N, int kind, bool visc, const KArgs<double> &a, int grid, cudaStream_t s);
cudaError_t prepare_2_f32(int N, bool visc);
cudaError_t prepare_2_f64(int N, bool visc);
cudaError_t prepare_3_f32(int N, bool visc);
cudaError_t prepare_3_f64(int N, bool visc);
}  // namespace frk

namespace fr {

thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

namespace {

// Carpenter-Kennedy five-stage fourth-order 2N-storage coefficients.
const double kLsA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kLsB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

constexpr int kPartialBlocks = 608;   // 4 x 152 SMs

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SlimMesh {         // what probe location needs from a mesh
    fr_mesh m;
};

}  // namespace
}  // namespace fr

struct fr_solver {
    int dim = 0, p = 0, N = 0, n_inst = 0;
    fr_config cfg{};
    bool fp64 = true, visc = false;
    int nsp = 0, nfp = 0, V = 0, MS = 0;
    int64_t E = 0, nb = 0, n_wall = 0, max_inst_e = 0;
    std::vector<int64_t> off, ne;
    cudaStream_t stream = nullptr;
    size_t rsz = 8;
    // device buffers
    char *U = nullptr, *R1 = nullptr, *R2 = nullptr, *RES = nullptr, *UF[2] = {nullptr, nullptr};
    char *FV = nullptr, *MET = nullptr, *NRM = nullptr, *BVREF = nullptr;
    int32_t *PART = nullptr, *BTAG = nullptr, *EINST = nullptr, *WALL = nullptr;
    double *stage64 = nullptr, *force_acc = nullptr, *partials = nullptr, *reduce_out = nullptr;
    frk::ProbeDesc *probes = nullptr;
    frk::ProbeAcc *pacc = nullptr;
    double *phist = nullptr;
    int n_probe = 0;
    std::vector<int> probe_inst;
    int parity = 0;
    int64_t steps_since_reset = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t launches_per_step = 0, last_launches = 0;
    std::vector<std::unique_ptr<fr_mesh>> host_meshes;   // for probe location
    // per-launch event pairs while fr_profile_steps runs
    bool profiling = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof;
    double ops_D1[frk::kMaxN * frk::kMaxN] = {}, ops_L[2 * frk::kMaxN] = {};
    double ops_GL[frk::kMaxN] = {}, ops_GR[frk::kMaxN] = {}, ops_W[frk::kMaxN] = {};
};

namespace fr {
namespace {

#define FR_CK(call)                                                                \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) {                                                   \
            fr::set_error(std::string("CUDA: ") + cudaGetErrorString(_e) + " at " + \
                          __FILE__ + ":" + std::to_string(__LINE__));              \
            return FR_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

struct Layout {
    size_t U, R1, R2, RES, UF0, UF1, FV, MET, NRM, PART, EINST, BTAG, BVREF, WALL, STAGE, PROBES,
        PACC, PHIST, FORCE, PART_SUMS, RED, total;
};

Layout make_layout(int dim, int nsp, int nfp, int64_t E, int64_t nb, int64_t nw, int64_t max_e,
                   int n_inst, bool fp64, bool visc) {
    const size_t rs = fp64 ? 8 : 4;
    const int V = dim + 2, MS = dim * dim + 1;
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + std::max<size_t>(bytes, 16)); return at; };
    const size_t st = (size_t)E * nsp * V * rs, fc = (size_t)E * nfp * V * rs;
    L.U = take(st);
    L.R1 = take(st);
    L.R2 = take(st);
    L.RES = take(st);
    L.UF0 = take(fc);
    L.UF1 = take(fc);
    L.FV = take(visc ? fc : 16);
    L.MET = take((size_t)E * nsp * MS * rs);
    L.NRM = take((size_t)E * nfp * dim * rs);
    L.PART = take((size_t)E * nfp * 4);
    L.EINST = take((size_t)E * 4);
    L.BTAG = take((size_t)nb * 4);
    L.BVREF = take((size_t)nb * dim * rs);
    L.WALL = take((size_t)nw * 4);
    L.STAGE = take((size_t)max_e * nsp * V * 8);
    L.PROBES = take(sizeof(frk::ProbeDesc) * kMaxProbes);
    L.PACC = take(sizeof(frk::ProbeAcc) * kMaxProbes);
    L.PHIST = take(sizeof(double) * kMaxProbes * frk::kHistLen);
    L.FORCE = take((size_t)n_inst * 3 * 8);
    L.PART_SUMS = take((size_t)kPartialBlocks * (2 * V + 1) * 8);
    L.RED = take((size_t)(V + 1) * 8);
    L.total = o;
    return L;
}

fr_status check_batch(fr_mesh *const *meshes, int n_inst, const fr_config *cfg) {
    if (!meshes || n_inst <= 0 || !cfg) { set_error("invalid solver arguments"); return FR_ERR_INVALID_ARG; }
    for (int i = 0; i < n_inst; ++i) {
        if (!meshes[i]) { set_error("null mesh in batch"); return FR_ERR_INVALID_ARG; }
        if (meshes[i]->dim != meshes[0]->dim || meshes[i]->p != meshes[0]->p) {
            set_error("all meshes of a batch must share dimension and degree");
            return FR_ERR_UNSUPPORTED;
        }
    }
    if (cfg->rk != FR_RK4 && cfg->rk != FR_LSRK45) { set_error("unknown rk scheme"); return FR_ERR_INVALID_ARG; }
    if (cfg->precision != FR_FP64 && cfg->precision != FR_FP32) { set_error("unknown precision"); return FR_ERR_INVALID_ARG; }
    if (cfg->flux != FR_FLUX_RUSANOV && cfg->flux != FR_FLUX_ROE) { set_error("unknown interface flux"); return FR_ERR_INVALID_ARG; }
    if (cfg->viscous_scheme != FR_VISC_BR2 && cfg->viscous_scheme != FR_VISC_LDG) { set_error("unknown viscous scheme"); return FR_ERR_INVALID_ARG; }
    if (!(cfg->gamma > 1.0) || !(cfg->rho_inf > 0.0) || !(cfg->p_inf > 0.0) || cfg->mu < 0.0 ||
        (cfg->viscous && !(cfg->prandtl > 0.0))) {
        set_error("invalid physical constants");
        return FR_ERR_INVALID_ARG;
    }
    return FR_OK;
}

void count_batch(fr_mesh *const *meshes, int n_inst, int64_t *E, int64_t *nb, int64_t *nw, int64_t *max_e) {
    *E = *nb = *nw = *max_e = 0;
    for (int i = 0; i < n_inst; ++i) {
        const fr_mesh *m = meshes[i];
        const int nfp = m->ref.nfp;
        *E += m->n_elem;
        *max_e = std::max(*max_e, m->n_elem);
        for (int64_t e = 0; e < m->n_elem; ++e) {
            bool wall = false;
            for (int f = 0; f < nfp; ++f) {
                const int32_t t = m->bctag[(size_t)e * nfp + f];
                if (t >= FR_TAG_WALL) ++*nb;
                if (t == FR_TAG_WALL) wall = true;
            }
            if (wall) ++*nw;
        }
    }
}

template <typename real>
void fill_args(const fr_solver *s, frk::KArgs<real> &a) {
    std::memset(&a, 0, sizeof(a));
    a.U = (real *)s->U;
    a.R1 = (real *)s->R1;
    a.R2 = (real *)s->R2;
    a.RES = (real *)s->RES;
    a.FV = (real *)s->FV;
    a.MET = (const real *)s->MET;
    a.NRM = (const real *)s->NRM;
    a.PART = s->PART;
    a.BTAG = s->BTAG;
    a.BVREF = (const real *)s->BVREF;
    a.EINST = s->EINST;
    a.gamma = (real)s->cfg.gamma;
    a.prandtl = (real)(s->cfg.prandtl > 0 ? s->cfg.prandtl : 1.0);
    a.mu = (real)(s->visc ? s->cfg.mu : 0.0);
    a.eta = (real)(s->cfg.br2_eta > 0 ? s->cfg.br2_eta : 2.0 * s->dim);
    a.rho_inf = (real)s->cfg.rho_inf;
    a.p_inf = (real)s->cfg.p_inf;
    a.dt = (real)s->cfg.dt;
    a.flux = s->cfg.flux;
    a.ldg = s->cfg.viscous_scheme == FR_VISC_LDG ? 1 : 0;
    a.ldg_beta = (real)s->cfg.ldg_beta;
    a.ldg_tau = (real)s->cfg.ldg_tau;
    a.probes = s->probes;
    a.pacc = s->pacc;
    a.phist = s->phist;
    a.n_probe = s->n_probe;
    a.force_acc = s->force_acc;
    a.partials = s->partials;
    a.reduce_out = s->reduce_out;
    a.n_partials = kPartialBlocks;
    a.stage64 = s->stage64;
    a.stage64_out = s->stage64;
    std::memcpy(a.opD1, s->ops_D1, sizeof(a.opD1));
    std::memcpy(a.opL, s->ops_L, sizeof(a.opL));
    std::memcpy(a.opGL, s->ops_GL, sizeof(a.opGL));
    std::memcpy(a.opGR, s->ops_GR, sizeof(a.opGR));
    std::memcpy(a.opW, s->ops_W, sizeof(a.opW));
}

// A launch description independent of the precision.
struct Launch {
    int kind = 0;
    int64_t elem0 = 0, n_elem = 0;
    const int32_t *elist = nullptr;
    int mode = 0, force = 0, integral_src = 0;
    double rk_a = 0, rk_b = 0, rk_c = 0;
    const void *UFin = nullptr;
    void *UFout = nullptr;
    int grid = 1;
};

template <typename real>
cudaError_t do_launch(const fr_solver *s, const Launch &L) {
    frk::KArgs<real> a;
    fill_args(s, a);
    a.elem0 = L.elem0;
    a.n_elem = L.n_elem;
    a.elist = L.elist;
    a.mode = L.mode;
    a.force = L.force;
    a.integral_src = L.integral_src;
    a.rk_a = (real)L.rk_a;
    a.rk_b = (real)L.rk_b;
    a.rk_c = (real)L.rk_c;
    a.UFin = (const real *)L.UFin;
    a.UFout = (real *)L.UFout;
    const bool visc = s->visc;
    if constexpr (std::is_same<real, float>::value) {
        return s->dim == 2 ? frk::launch_2_f32(s->N, L.kind, visc, a, L.grid, s->stream)
                           : frk::launch_3_f32(s->N, L.kind, visc, a, L.grid, s->stream);
    } else {
        return s->dim == 2 ? frk::launch_2_f64(s->N, L.kind, visc, a, L.grid, s->stream)
                           : frk::launch_3_f64(s->N, L.kind, visc, a, L.grid, s->stream);
    }
}

// profiling kinds of fr_profile_steps
enum ProfKind { P_FLUX = 0, P_GRAD = 1, P_PROBE = 2, P_FORCE = 3, P_OTHER = 4 };

int prof_kind(const Launch &L) {
    if (L.kind == frk::K_FLUX) return P_FLUX;
    if (L.kind == frk::K_GRAD) return L.force ? P_FORCE : P_GRAD;
    if (L.kind == frk::K_PROBE) return P_PROBE;
    return P_OTHER;
}

cudaError_t launch(const fr_solver *s, const Launch &L) {
    if (s->profiling) {
        cudaEvent_t a, b;
        cudaError_t e = cudaEventCreate(&a);
        if (e != cudaSuccess) return e;
        e = cudaEventCreate(&b);
        if (e != cudaSuccess) return e;
        cudaEventRecord(a, s->stream);
        e = s->fp64 ? do_launch<double>(s, L) : do_launch<float>(s, L);
        cudaEventRecord(b, s->stream);
        const_cast<fr_solver *>(s)->prof.push_back({prof_kind(L), {a, b}});
        return e;
    }
    return s->fp64 ? do_launch<double>(s, L) : do_launch<float>(s, L);
}

int grid_for(int64_t items) {
    int64_t g = (items + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, kPartialBlocks));
}

// One RK step starting from face-buffer parity p0; returns the launches issued.
fr_status enqueue_step(fr_solver *s, int p0, int64_t *n_launch) {
    int par = p0;
    int64_t cnt = 0;
    const int stages = s->cfg.rk == FR_RK4 ? 4 : 5;
    const double dt = s->cfg.dt;
    for (int st = 0; st < stages; ++st) {
        if (s->visc) {
            Launch g;
            g.kind = frk::K_GRAD;
            g.n_elem = s->E;
            g.UFin = s->UF[par];
            FR_CK(launch(s, g));
            ++cnt;
        }
        Launch f;
        f.kind = frk::K_FLUX;
        f.n_elem = s->E;
        f.UFin = s->UF[par];
        f.UFout = s->UF[par ^ 1];
        if (s->cfg.rk == FR_LSRK45) {
            f.mode = st == 0 ? frk::M_LSRK_FIRST : frk::M_LSRK;
            f.rk_a = kLsA[st];
            f.rk_b = kLsB[st];
        } else {
            const int modes[4] = {frk::M_RK4_1, frk::M_RK4_2, frk::M_RK4_3, frk::M_RK4_4};
            const double cs[4] = {0.5 * dt, 0.5 * dt, dt, dt / 6.0};
            f.mode = modes[st];
            f.rk_c = cs[st];
        }
        FR_CK(launch(s, f));
        ++cnt;
        par ^= 1;
    }
    if (s->n_probe > 0) {
        Launch pr;
        pr.kind = frk::K_PROBE;
        FR_CK(launch(s, pr));
        ++cnt;
    }
    if (s->n_wall > 0) {
        Launch fo;
        fo.kind = frk::K_GRAD;
        fo.force = 1;
        fo.elist = s->WALL;
        fo.n_elem = s->n_wall;
        fo.UFin = s->UF[par];
        FR_CK(launch(s, fo));
        ++cnt;
    }
    *n_launch = cnt;
    return FR_OK;
}

void drop_graphs(fr_solver *s) {
    for (int i = 0; i < 2; ++i)
        if (s->graph[i]) {
            cudaGraphExecDestroy(s->graph[i]);
            s->graph[i] = nullptr;
        }
}

fr_status check_inst(fr_solver *s, int inst) {
    if (!s) { set_error("null solver"); return FR_ERR_INVALID_ARG; }
    if (inst < 0 || inst >= s->n_inst) { set_error("instance index out of range"); return FR_ERR_INVALID_ARG; }
    return FR_OK;
}

// residual (or J * residual) of one instance into RES
fr_status residual_into_res(fr_solver *s, int inst, int mode) {
    if (s->visc) {
        Launch g;
        g.kind = frk::K_GRAD;
        g.elem0 = s->off[inst];
        g.n_elem = s->ne[inst];
        g.UFin = s->UF[s->parity];
        FR_CK(launch(s, g));
    }
    Launch f;
    f.kind = frk::K_FLUX;
    f.elem0 = s->off[inst];
    f.n_elem = s->ne[inst];
    f.UFin = s->UF[s->parity];
    f.mode = mode;
    FR_CK(launch(s, f));
    return FR_OK;
}

fr_status reduce_integral(fr_solver *s, int inst, int src, double *out_sums, double *out_bad) {
    FR_CK(cudaMemsetAsync(s->partials, 0, (size_t)kPartialBlocks * (2 * s->V + 1) * 8, s->stream));
    Launch in;
    in.kind = frk::K_INTEGRAL;
    in.elem0 = s->off[inst];
    in.n_elem = s->ne[inst];
    in.integral_src = src;
    in.grid = kPartialBlocks;
    FR_CK(launch(s, in));
    Launch rd;
    rd.kind = frk::K_REDUCE;
    FR_CK(launch(s, rd));
    std::vector<double> h(s->V + 1);
    FR_CK(cudaMemcpyAsync(h.data(), s->reduce_out, h.size() * 8, cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    for (int v = 0; v < s->V; ++v) out_sums[v] = h[v];
    if (out_bad) *out_bad = h[s->V];
    return FR_OK;
}

}  // namespace
}  // namespace fr

using namespace fr;

extern "C" const char *fr_last_error(void) { return fr::g_last_error.c_str(); }

extern "C" size_t fr_workspace_bytes(fr_mesh *const *meshes, int n_inst, const fr_config *cfg) {
    if (check_batch(meshes, n_inst, cfg) != FR_OK) return 0;
    int64_t E, nb, nw, mx;
    count_batch(meshes, n_inst, &E, &nb, &nw, &mx);
    const fr_mesh *m = meshes[0];
    Layout L = make_layout(m->dim, m->ref.nsp, m->ref.nfp, E, nb, nw, mx, n_inst,
                           cfg->precision == FR_FP64, cfg->viscous != 0);
    return L.total;
}

namespace {
template <typename real>
void to_real(std::vector<char> &dst, const std::vector<double> &src) {
    dst.resize(src.size() * sizeof(real));
    real *d = reinterpret_cast<real *>(dst.data());
    for (size_t i = 0; i < src.size(); ++i) d[i] = (real)src[i];
}
}  // namespace

extern "C" fr_status fr_solver_create(fr_solver **out, fr_mesh *const *meshes, int n_inst,
                                      const fr_config *cfg, void *workspace, size_t ws_bytes,
                                      void *stream) {
    if (!out) { set_error("null output pointer"); return FR_ERR_INVALID_ARG; }
    *out = nullptr;
    fr_status st = check_batch(meshes, n_inst, cfg);
    if (st != FR_OK) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        set_error("workspace must be a non-null device pointer aligned to 256 bytes");
        return FR_ERR_WORKSPACE;
    }
    auto s = std::make_unique<fr_solver>();
    const fr_mesh *m0 = meshes[0];
    s->dim = m0->dim;
    s->p = m0->p;
    s->N = m0->p + 1;
    s->n_inst = n_inst;
    s->cfg = *cfg;
    s->fp64 = cfg->precision == FR_FP64;
    s->visc = cfg->viscous != 0;
    s->nsp = m0->ref.nsp;
    s->nfp = m0->ref.nfp;
    s->V = s->dim + 2;
    s->MS = s->dim * s->dim + 1;
    s->rsz = s->fp64 ? 8 : 4;
    s->stream = (cudaStream_t)stream;
    count_batch(meshes, n_inst, &s->E, &s->nb, &s->n_wall, &s->max_inst_e);
    if (s->E * (int64_t)s->nfp >= ((int64_t)1 << 31)) {
        set_error("batch too large for 32-bit flux-point indices");
        return FR_ERR_UNSUPPORTED;
    }
    Layout L = make_layout(s->dim, s->nsp, s->nfp, s->E, s->nb, s->n_wall, s->max_inst_e, n_inst,
                           s->fp64, s->visc);
    if (ws_bytes < L.total) {
        set_error("workspace too small: need " + std::to_string(L.total) + " bytes");
        return FR_ERR_WORKSPACE;
    }
    char *w = (char *)workspace;
    s->U = w + L.U; s->R1 = w + L.R1; s->R2 = w + L.R2; s->RES = w + L.RES;
    s->UF[0] = w + L.UF0; s->UF[1] = w + L.UF1; s->FV = w + L.FV;
    s->MET = w + L.MET; s->NRM = w + L.NRM; s->BVREF = w + L.BVREF;
    s->PART = (int32_t *)(w + L.PART); s->EINST = (int32_t *)(w + L.EINST);
    s->BTAG = (int32_t *)(w + L.BTAG); s->WALL = (int32_t *)(w + L.WALL);
    s->stage64 = (double *)(w + L.STAGE);
    s->probes = (frk::ProbeDesc *)(w + L.PROBES);
    s->pacc = (frk::ProbeAcc *)(w + L.PACC);
    s->phist = (double *)(w + L.PHIST);
    s->force_acc = (double *)(w + L.FORCE);
    s->partials = (double *)(w + L.PART_SUMS);
    s->reduce_out = (double *)(w + L.RED);

    const RefElem &r = m0->ref;
    for (int i = 0; i < s->N; ++i) {
        for (int mm = 0; mm < s->N; ++mm) s->ops_D1[i * frk::kMaxN + mm] = r.D1[i][mm];
        s->ops_L[i] = r.lend[0][i];
        s->ops_L[frk::kMaxN + i] = r.lend[1][i];
        s->ops_GL[i] = r.dgL[i];
        s->ops_GR[i] = r.dgR[i];
        s->ops_W[i] = r.w[i];
    }

    // host tables, FP64 first, cast once
    const int dim = s->dim, nsp = s->nsp, nfp = s->nfp, MS = s->MS;
    std::vector<double> met((size_t)s->E * nsp * MS), nrm((size_t)s->E * nfp * dim),
        bvref((size_t)std::max<int64_t>(s->nb, 1) * dim, 0.0);
    std::vector<int32_t> part((size_t)s->E * nfp), einst(s->E), btag(std::max<int64_t>(s->nb, 1)),
        wall(std::max<int64_t>(s->n_wall, 1));
    int64_t off = 0, b = 0, nwl = 0;
    for (int i = 0; i < n_inst; ++i) {
        const fr_mesh *m = meshes[i];
        s->off.push_back(off);
        s->ne.push_back(m->n_elem);
        for (int64_t e = 0; e < m->n_elem; ++e) {
            const int64_t ge = off + e;
            einst[ge] = i;
            for (int sp = 0; sp < nsp; ++sp) {
                const size_t src = (size_t)e * nsp + sp;
                for (int kk = 0; kk < dim * dim; ++kk)
                    met[((size_t)ge * nsp + sp) * MS + kk] = m->S[src * dim * dim + kk];
                met[((size_t)ge * nsp + sp) * MS + dim * dim] = 1.0 / m->J[src];
            }
            bool has_wall = false;
            for (int f = 0; f < nfp; ++f) {
                const size_t lf = (size_t)e * nfp + f;
                for (int d = 0; d < dim; ++d) nrm[((size_t)ge * nfp + f) * dim + d] = m->nrm[lf * dim + d];
                const int64_t pt = m->partner[lf];
                if (pt >= 0) {
                    part[(size_t)ge * nfp + f] = (int32_t)(off * nfp + pt);
                } else {
                    const int32_t tag = m->bctag[lf];
                    part[(size_t)ge * nfp + f] = (int32_t)(-1 - b);
                    btag[b] = tag;
                    // reference velocity at this point (tanh profile on inflow)
                    double prof = 1.0;
                    if (tag == FR_TAG_INFLOW && cfg->inflow_delta > 0.0)
                        prof = std::tanh(3.0 * (m->x_fp[lf * dim + 1] - cfg->inflow_ywall) / cfg->inflow_delta);
                    for (int d = 0; d < dim; ++d) bvref[(size_t)b * dim + d] = cfg->v_inf[d] * prof;
                    if (tag == FR_TAG_WALL) has_wall = true;
                    ++b;
                }
            }
            if (has_wall) wall[nwl++] = (int32_t)ge;
        }
        off += m->n_elem;
        // slim host copy for probe location
        auto hm = std::make_unique<fr_mesh>();
        hm->dim = m->dim; hm->p = m->p; hm->q = m->q; hm->ref = m->ref; hm->n_elem = m->n_elem;
        hm->nodes = m->nodes;
        s->host_meshes.push_back(std::move(hm));
    }
    std::vector<char> tmp;
    cudaStream_t cs = s->stream;
    auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(cs);
    };
    if (s->fp64) {
        FR_CK(up(s->MET, met.data(), met.size() * 8));
        FR_CK(up(s->NRM, nrm.data(), nrm.size() * 8));
        FR_CK(up(s->BVREF, bvref.data(), (size_t)s->nb * dim * 8));
    } else {
        to_real<float>(tmp, met); FR_CK(up(s->MET, tmp.data(), tmp.size()));
        to_real<float>(tmp, nrm); FR_CK(up(s->NRM, tmp.data(), tmp.size()));
        to_real<float>(tmp, bvref); FR_CK(up(s->BVREF, tmp.data(), (size_t)s->nb * dim * 4));
    }
    FR_CK(up(s->PART, part.data(), part.size() * 4));
    FR_CK(up(s->EINST, einst.data(), einst.size() * 4));
    if (s->nb > 0) FR_CK(up(s->BTAG, btag.data(), (size_t)s->nb * 4));
    if (s->n_wall > 0) FR_CK(up(s->WALL, wall.data(), (size_t)s->n_wall * 4));
    const size_t st_bytes = (size_t)s->E * nsp * s->V * s->rsz, fc_bytes = (size_t)s->E * nfp * s->V * s->rsz;
    FR_CK(cudaMemsetAsync(s->U, 0, st_bytes, cs));
    FR_CK(cudaMemsetAsync(s->R1, 0, st_bytes, cs));
    FR_CK(cudaMemsetAsync(s->R2, 0, st_bytes, cs));
    FR_CK(cudaMemsetAsync(s->RES, 0, st_bytes, cs));
    FR_CK(cudaMemsetAsync(s->UF[0], 0, fc_bytes, cs));
    FR_CK(cudaMemsetAsync(s->UF[1], 0, fc_bytes, cs));
    if (s->visc) FR_CK(cudaMemsetAsync(s->FV, 0, fc_bytes, cs));
    FR_CK(cudaMemsetAsync(s->pacc, 0, sizeof(frk::ProbeAcc) * kMaxProbes, cs));
    FR_CK(cudaMemsetAsync(s->force_acc, 0, (size_t)n_inst * 3 * 8, cs));
    FR_CK(cudaStreamSynchronize(cs));
    cudaError_t pe;
    if (dim == 2) pe = s->fp64 ? frk::prepare_2_f64(s->N, s->visc) : frk::prepare_2_f32(s->N, s->visc);
    else pe = s->fp64 ? frk::prepare_3_f64(s->N, s->visc) : frk::prepare_3_f32(s->N, s->visc);
    FR_CK(pe);
    *out = s.release();
    return FR_OK;
}

extern "C" void fr_solver_destroy(fr_solver *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    drop_graphs(s);
    delete s;
}

extern "C" fr_status fr_set_state(fr_solver *s, int inst, const double *u) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!u) { set_error("null state"); return FR_ERR_INVALID_ARG; }
    const size_t n = (size_t)s->ne[inst] * s->nsp * s->V;
    FR_CK(cudaMemcpyAsync(s->stage64, u, n * 8, cudaMemcpyHostToDevice, s->stream));
    Launch c;
    c.kind = frk::K_TO_REAL;
    c.elem0 = s->off[inst];
    c.n_elem = s->ne[inst];
    c.grid = grid_for((int64_t)n);
    FR_CK(launch(s, c));
    Launch in;
    in.kind = frk::K_INTERP;
    in.elem0 = s->off[inst];
    in.n_elem = s->ne[inst];
    in.UFout = s->UF[s->parity];
    FR_CK(launch(s, in));
    FR_CK(cudaStreamSynchronize(s->stream));
    return FR_OK;
}

static fr_status copy_out(fr_solver *s, int inst, int src, double *u) {
    const size_t n = (size_t)s->ne[inst] * s->nsp * s->V;
    Launch c;
    c.kind = frk::K_TO_F64;
    c.elem0 = s->off[inst];
    c.n_elem = s->ne[inst];
    c.integral_src = src;
    c.grid = grid_for((int64_t)n);
    FR_CK(launch(s, c));
    FR_CK(cudaMemcpyAsync(u, s->stage64, n * 8, cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    return FR_OK;
}

extern "C" fr_status fr_get_state(fr_solver *s, int inst, double *u) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!u) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    return copy_out(s, inst, 0, u);
}

extern "C" fr_status fr_residual(fr_solver *s, int inst, double *r) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!r) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    st = residual_into_res(s, inst, frk::M_RESIDUAL);
    if (st != FR_OK) return st;
    return copy_out(s, inst, 1, r);
}

extern "C" fr_status fr_rk_step(fr_solver *s, int n_steps) {
    if (!s || n_steps < 0) { set_error("invalid fr_rk_step arguments"); return FR_ERR_INVALID_ARG; }
    const int stages = s->cfg.rk == FR_RK4 ? 4 : 5;
    int64_t total = 0;
    for (int it = 0; it < n_steps; ++it) {
        const int p0 = s->parity;
        if (s->stream) {
            if (!s->graph[p0]) {
                cudaGraph_t g;
                FR_CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
                int64_t cnt = 0;
                fr_status st = enqueue_step(s, p0, &cnt);
                cudaError_t ce = cudaStreamEndCapture(s->stream, &g);
                if (st != FR_OK) return st;
                FR_CK(ce);
                cudaError_t ie = cudaGraphInstantiate(&s->graph[p0], g, 0);
                cudaGraphDestroy(g);
                FR_CK(ie);
                s->launches_per_step = cnt;
            }
            FR_CK(cudaGraphLaunch(s->graph[p0], s->stream));
            total += s->launches_per_step;
        } else {
            int64_t cnt = 0;
            fr_status st = enqueue_step(s, p0, &cnt);
            if (st != FR_OK) return st;
            total += cnt;
        }
        s->parity = (stages % 2) ? p0 ^ 1 : p0;
        ++s->steps_since_reset;
    }
    s->last_launches = total;
    return FR_OK;
}

extern "C" int64_t fr_last_launch_count(const fr_solver *s) { return s ? s->last_launches : -1; }

extern "C" fr_status fr_profile_steps(fr_solver *s, int n_steps, double *ms, int64_t *count) {
    if (!s || n_steps <= 0 || !ms || !count) { set_error("invalid fr_profile_steps arguments"); return FR_ERR_INVALID_ARG; }
    const int stages = s->cfg.rk == FR_RK4 ? 4 : 5;
    s->prof.clear();
    s->profiling = true;
    fr_status st = FR_OK;
    for (int it = 0; it < n_steps && st == FR_OK; ++it) {
        int64_t cnt = 0;
        st = enqueue_step(s, s->parity, &cnt);
        s->parity = (stages % 2) ? s->parity ^ 1 : s->parity;
        ++s->steps_since_reset;
    }
    s->profiling = false;
    cudaError_t se = cudaStreamSynchronize(s->stream);
    for (int k = 0; k < 5; ++k) { ms[k] = 0.0; count[k] = 0; }
    for (auto &pe : s->prof) {
        float t = 0.f;
        if (se == cudaSuccess) cudaEventElapsedTime(&t, pe.second.first, pe.second.second);
        ms[pe.first] += t;
        count[pe.first] += 1;
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    s->prof.clear();
    for (int k = 0; k < 5; ++k)
        if (count[k]) ms[k] /= (double)count[k];
    if (st != FR_OK) return st;
    FR_CK(se);
    return FR_OK;
}

extern "C" fr_status fr_probe_add(fr_solver *s, int inst, const double *x, int *probe_id) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!x || !probe_id) { set_error("null argument"); return FR_ERR_INVALID_ARG; }
    if (s->n_probe >= kMaxProbes) { set_error("too many probes"); return FR_ERR_INVALID_ARG; }
    const fr_mesh &m = *s->host_meshes[inst];
    int64_t e;
    double xi[3] = {0, 0, 0};
    if (!mesh_locate(m, x, &e, xi)) { set_error("probe point outside the mesh"); return FR_ERR_INVALID_ARG; }
    frk::ProbeDesc d;
    std::memset(&d, 0, sizeof(d));
    d.elem = s->off[inst] + e;
    d.inst = inst;
    ref_interp(m.ref, xi, d.w);
    const int id = s->n_probe;
    FR_CK(cudaMemcpyAsync(&s->probes[id], &d, sizeof(d), cudaMemcpyHostToDevice, s->stream));
    FR_CK(cudaMemsetAsync(&s->pacc[id], 0, sizeof(frk::ProbeAcc), s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    s->n_probe += 1;
    s->probe_inst.push_back(inst);
    drop_graphs(s);   // the captured step must include the new observer
    *probe_id = id;
    return FR_OK;
}

static fr_status read_acc(fr_solver *s, int id, frk::ProbeAcc *a) {
    if (!s || id < 0 || id >= s->n_probe) { set_error("invalid probe id"); return FR_ERR_INVALID_ARG; }
    FR_CK(cudaMemcpyAsync(a, &s->pacc[id], sizeof(*a), cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    return FR_OK;
}

extern "C" fr_status fr_probe_pressure(fr_solver *s, int probe_id, double *p_latest) {
    if (!p_latest) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    frk::ProbeAcc a;
    fr_status st = read_acc(s, probe_id, &a);
    if (st != FR_OK) return st;
    *p_latest = a.last;
    return FR_OK;
}

extern "C" fr_status fr_probe_stats(fr_solver *s, int probe_id, double *out4) {
    if (!out4) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    frk::ProbeAcc a;
    fr_status st = read_acc(s, probe_id, &a);
    if (st != FR_OK) return st;
    out4[0] = a.count;
    out4[1] = a.count > 0 ? (a.sum + a.sum_c) / a.count : 0.0;
    out4[2] = a.sq0 + a.sq0_c;
    out4[3] = a.m2 + a.m2_c;
    return FR_OK;
}

extern "C" fr_status fr_probe_history(fr_solver *s, int probe_id, double *out, int max_n, int *n_out) {
    if (!out || !n_out || max_n < 0) { set_error("invalid fr_probe_history arguments"); return FR_ERR_INVALID_ARG; }
    frk::ProbeAcc a;
    fr_status st = read_acc(s, probe_id, &a);
    if (st != FR_OK) return st;
    const int64_t count = (int64_t)a.count;
    const int64_t keep = std::min<int64_t>(std::min<int64_t>(count, frk::kHistLen), max_n);
    const double *ring = s->phist + (size_t)probe_id * frk::kHistLen;
    // the most recent `keep` samples, oldest first: ring index (count - keep + i) % len
    const int64_t first = (count - keep) % frk::kHistLen;
    const int64_t n1 = std::min<int64_t>(keep, frk::kHistLen - first);
    if (n1 > 0) FR_CK(cudaMemcpyAsync(out, ring + first, n1 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (keep > n1)
        FR_CK(cudaMemcpyAsync(out + n1, ring, (keep - n1) * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    *n_out = (int)keep;
    return FR_OK;
}

extern "C" fr_status fr_probe_reset(fr_solver *s) {
    if (!s) { set_error("null solver"); return FR_ERR_INVALID_ARG; }
    FR_CK(cudaMemsetAsync(s->pacc, 0, sizeof(frk::ProbeAcc) * kMaxProbes, s->stream));
    FR_CK(cudaMemsetAsync(s->force_acc, 0, (size_t)s->n_inst * 3 * 8, s->stream));
    s->steps_since_reset = 0;
    return FR_OK;
}

extern "C" fr_status fr_oaspl(fr_solver *s, const int *ids, int n, double p_ref, double p_scale,
                              int mean_mode, double *oaspl_db) {
    if (!s || !ids || n <= 0 || !oaspl_db || !(p_ref > 0) || (mean_mode != 0 && mean_mode != 1)) {
        set_error("invalid fr_oaspl arguments");
        return FR_ERR_INVALID_ARG;
    }
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        frk::ProbeAcc a;
        fr_status st = read_acc(s, ids[i], &a);
        if (st != FR_OK) return st;
        if (a.count <= 0) { set_error("probe has no samples"); return FR_ERR_INVALID_ARG; }
        const double ss = mean_mode == 0 ? a.sq0 + a.sq0_c : a.m2 + a.m2_c;
        acc += std::sqrt(std::max(ss, 0.0) / a.count);
    }
    const double prms = acc / n;
    *oaspl_db = prms == 0.0 ? -INFINITY : 20.0 * std::log10(p_scale * prms / p_ref);
    return FR_OK;
}

extern "C" fr_status fr_forces(fr_solver *s, int inst, double *mean_force) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!mean_force) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    double h[3];
    FR_CK(cudaMemcpyAsync(h, s->force_acc + (size_t)inst * 3, 24, cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    const double n = (double)std::max<int64_t>(s->steps_since_reset, 1);
    for (int d = 0; d < s->dim; ++d) mean_force[d] = h[d] / n;
    return FR_OK;
}

extern "C" fr_status fr_conservation(fr_solver *s, int inst, double *sums) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!sums) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    st = residual_into_res(s, inst, frk::M_RESIDUAL_J);
    if (st != FR_OK) return st;
    return reduce_integral(s, inst, 1, sums, nullptr);
}

extern "C" fr_status fr_integral(fr_solver *s, int inst, double *sums, int64_t *n_nonfinite) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!sums) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    double bad = 0;
    st = reduce_integral(s, inst, 0, sums, &bad);
    if (n_nonfinite) *n_nonfinite = (int64_t)bad;
    if (st == FR_OK && bad > 0) { set_error("non-finite values in the state"); return FR_ERR_NONFINITE; }
    return st;
}

// --------------------------------------------------------------------------
// Allocation-free integral (fr_integral_static)
//
// Same result as fr_integral, but the per-block partial sums and the final
// sums live in a file-scope device array instead of the solver's workspace.
// The array is part of the loaded module: every GPU that loads libfr.so holds
// it until the process exits, and all calls share it.
// --------------------------------------------------------------------------
namespace fr {
namespace {

constexpr int kStaticBlocks = 1024;                 // partial-sum slots
constexpr int kStaticThreads = 256;
constexpr int kStaticItemsPerThread = 8;
constexpr int64_t kStaticMaxItems = (int64_t)kStaticBlocks * kStaticThreads * kStaticItemsPerThread;
constexpr int kStaticSlotsPerBlock = 2 * 5 + 1;      // sum, compensation (V <= 5), non-finite count
constexpr size_t kStaticDoubles = (size_t)kStaticBlocks * kStaticSlotsPerBlock + 8;

__device__ __align__(256) double g_static_scratch[kStaticDoubles];

std::mutex g_static_mu;
double *g_static_ptr[64] = {};   // device address of g_static_scratch, per device

// Device address of the scratch array on the current device.  Looked up once
// per device (cudaGetSymbolAddress), with that device current.
fr_status static_scratch(double **out) {
    int dev = 0;
    FR_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device index out of range"); return FR_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        FR_CK(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_static_ptr[dev];
    return FR_OK;
}

template <typename real>
cudaError_t launch_static(const fr_solver *s, int kind, int inst, int grid, double *scratch) {
    frk::KArgs<real> a;
    fill_args(s, a);
    a.elem0 = s->off[inst];
    a.n_elem = s->ne[inst];
    a.integral_src = 0;
    a.partials = scratch;
    a.n_partials = grid;
    a.reduce_out = scratch + (size_t)kStaticBlocks * kStaticSlotsPerBlock;
    if constexpr (std::is_same<real, float>::value) {
        return s->dim == 2 ? frk::launch_2_f32(s->N, kind, s->visc, a, grid, s->stream)
                           : frk::launch_3_f32(s->N, kind, s->visc, a, grid, s->stream);
    } else {
        return s->dim == 2 ? frk::launch_2_f64(s->N, kind, s->visc, a, grid, s->stream)
                           : frk::launch_3_f64(s->N, kind, s->visc, a, grid, s->stream);
    }
}

}  // namespace
}  // namespace fr

extern "C" fr_status fr_integral_static(fr_solver *s, int inst, double *sums, int64_t *n_nonfinite) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!sums) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    const int64_t items = s->ne[inst] * (int64_t)s->nsp;
    if (items > fr::kStaticMaxItems) {
        set_error("fr_integral_static: instance has " + std::to_string(items) +
                  " solution points, more than the static scratch serves (" +
                  std::to_string(fr::kStaticMaxItems) + "); use fr_integral");
        return FR_ERR_INVALID_ARG;
    }
    double *scratch = nullptr;
    st = fr::static_scratch(&scratch);
    if (st != FR_OK) return st;
    const int per_block = fr::kStaticThreads * fr::kStaticItemsPerThread;
    const int grid = (int)std::max<int64_t>(1, (items + per_block - 1) / per_block);
    // every block writes all of its slots; the result slots are cleared anyway
    FR_CK(cudaMemsetAsync(scratch, 0, fr::kStaticDoubles * sizeof(double), s->stream));
    FR_CK(s->fp64 ? fr::launch_static<double>(s, frk::K_INTEGRAL, inst, grid, scratch)
                  : fr::launch_static<float>(s, frk::K_INTEGRAL, inst, grid, scratch));
    FR_CK(s->fp64 ? fr::launch_static<double>(s, frk::K_REDUCE, inst, grid, scratch)
                  : fr::launch_static<float>(s, frk::K_REDUCE, inst, grid, scratch));
    double h[6] = {0, 0, 0, 0, 0, 0};
    FR_CK(cudaMemcpyAsync(h, scratch + (size_t)fr::kStaticBlocks * fr::kStaticSlotsPerBlock,
                          (size_t)(s->V + 1) * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    for (int v = 0; v < s->V; ++v) sums[v] = h[v];
    if (n_nonfinite) *n_nonfinite = (int64_t)h[s->V];
    if (h[s->V] > 0) { set_error("non-finite values in the state"); return FR_ERR_NONFINITE; }
    return FR_OK;
}
