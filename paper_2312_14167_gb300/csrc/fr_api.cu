// C ABI of the FR library (include/fr.h): batch solver object, workspace
// carving, CUDA-graph replay of the RK step, probes, OASPL and the FP64
// reductions.  Kernels live in fr_kernels.cuh, instantiated per dimension and
// precision in fr_k{2,3}_{f32,f64}.cu.
//
// The elements of a batch are grouped by polynomial degree; each group has
// its own element tables and kernels (one template instance per degree).
// Faces joining two degrees (meshes built by fr_mesh_create_varp) are
// coupled by the mortar kernels between the group kernels of each stage.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
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
cudaError_t mortar_2_f32(const MArgs<float> &a, cudaStream_t s);
cudaError_t mortar_2_f64(const MArgs<double> &a, cudaStream_t s);
cudaError_t mortar_3_f32(const MArgs<float> &a, cudaStream_t s);
cudaError_t mortar_3_f64(const MArgs<double> &a, cudaStream_t s);
}  // namespace frk

namespace fr {

thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

// NVTX range around a public call (visible to nsys / ncu; free without a tool)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

namespace {

// Carpenter-Kennedy five-stage fourth-order 2N-storage coefficients.
const double kLsA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kLsB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

constexpr int kPartialBlocks = 608;   // 4 x 152 SMs

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// the uniform-degree parts of a mesh (a uniform mesh is its own part)
std::vector<const fr_mesh *> parts_of(const fr_mesh *m) {
    std::vector<const fr_mesh *> out;
    if (m->parts.empty()) out.push_back(m);
    else
        for (auto &p : m->parts) out.push_back(p.get());
    return out;
}

bool is_boundary_tag(int32_t t) { return t >= FR_TAG_WALL && t <= FR_TAG_OUTFLOW; }

}  // namespace

// One degree group of a batch: all elements of that degree, instance after
// instance, each instance's elements in their mesh order.
struct Group {
    int p = 0, N = 0, nsp = 0, nfp = 0, nfpf = 0;
    int64_t E = 0, n_wall = 0;
    // outbox rows of mortar faces follow the E * nfp flux points: first the
    // faces where this group is the lower-degree side, then the others
    int64_t fp_real = 0, n_box_lo = 0, n_box = 0;
    std::vector<int64_t> off, ne;            // per instance
    char *U = nullptr, *R1 = nullptr, *R2 = nullptr, *RES = nullptr, *UF[2] = {nullptr, nullptr};
    char *FV = nullptr, *MET = nullptr, *NRM = nullptr, *MFLUX = nullptr;
    int32_t *PART = nullptr, *EINST = nullptr, *WALL = nullptr;
    int n_probe = 0;
    RefElem ref;
};

// Sizes of a batch, shared by fr_workspace_bytes and fr_solver_create.
struct Plan {
    int dim = 0, G = 0;
    int group_of_degree[kMaxN] = {-1, -1, -1, -1, -1};
    int degree[frk::kMaxGroups] = {};
    int64_t E[frk::kMaxGroups] = {}, n_wall[frk::kMaxGroups] = {};
    int64_t box_lo[frk::kMaxGroups] = {}, box_hi[frk::kMaxGroups] = {};
    int64_t nb = 0, stage_doubles = 0, n_mortar = 0;
    std::map<int, int64_t> mat_off;   // (p_lo, p_hi, orient) -> offset in the matrix table
    int64_t mat_reals = 0;
};

int mat_key(int plo, int phi, int o) { return (plo * 8 + phi) * 8 + o; }

}  // namespace fr

struct fr_solver {
    int dim = 0, n_inst = 0, V = 0, MS = 0;
    fr_config cfg{};
    bool fp64 = true, visc = false;
    std::vector<fr::Group> grp;
    int64_t nb = 0;
    cudaStream_t stream = nullptr;
    size_t rsz = 8;
    // per instance: number of solution points; for instances spread over
    // several groups, the group, in-group index and host offset of every element
    std::vector<int64_t> inst_nsp;
    std::vector<std::vector<int32_t>> egroup;
    std::vector<std::vector<int64_t>> elocal, esp;
    // mortar faces (sorted by instance) and their operators
    int64_t n_mortar = 0;
    std::vector<int64_t> moff, mcnt;
    frk::MortarFace *MORT = nullptr;
    char *MATS = nullptr;
    // shared device buffers
    char *BVREF = nullptr;
    int32_t *BTAG = nullptr;
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

fr_status check_batch(fr_mesh *const *meshes, int n_inst, const fr_config *cfg) {
    if (!meshes || n_inst <= 0 || !cfg) { set_error("invalid solver arguments"); return FR_ERR_INVALID_ARG; }
    for (int i = 0; i < n_inst; ++i) {
        if (!meshes[i]) { set_error("null mesh in batch"); return FR_ERR_INVALID_ARG; }
        if (meshes[i]->dim != meshes[0]->dim) {
            set_error("all meshes of a batch must share the dimension");
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

Plan make_plan(fr_mesh *const *meshes, int n_inst) {
    Plan P;
    P.dim = meshes[0]->dim;
    const int V = P.dim + 2;
    bool present[kMaxN] = {};
    for (int i = 0; i < n_inst; ++i)
        for (const fr_mesh *pm : parts_of(meshes[i])) present[pm->p] = true;
    for (int d = 0; d < kMaxN; ++d)
        if (present[d]) { P.group_of_degree[d] = P.G; P.degree[P.G] = d; ++P.G; }
    for (int i = 0; i < n_inst; ++i) {
        const fr_mesh *m = meshes[i];
        int64_t nsp_inst = 0;
        for (const fr_mesh *pm : parts_of(m)) {
            const int g = P.group_of_degree[pm->p];
            const int nfp = pm->ref.nfp;
            P.E[g] += pm->n_elem;
            nsp_inst += pm->n_elem * pm->ref.nsp;
            for (int64_t e = 0; e < pm->n_elem; ++e) {
                bool wall = false;
                for (int f = 0; f < nfp; ++f) {
                    const int32_t t = pm->bctag[(size_t)e * nfp + f];
                    if (is_boundary_tag(t)) ++P.nb;
                    if (t == FR_TAG_WALL) wall = true;
                }
                if (wall) ++P.n_wall[g];
            }
        }
        P.stage_doubles = std::max(P.stage_doubles, nsp_inst * V);
        for (const MortarLink &L : m->mortars) {
            const fr_mesh *lo = m->parts[L.part_lo].get(), *hi = m->parts[L.part_hi].get();
            P.box_lo[P.group_of_degree[lo->p]] += lo->ref.nfpf;
            P.box_hi[P.group_of_degree[hi->p]] += hi->ref.nfpf;
            ++P.n_mortar;
            const int key = mat_key(lo->p, hi->p, L.orient);
            if (!P.mat_off.count(key)) {
                P.mat_off[key] = P.mat_reals;
                P.mat_reals += 2 * (int64_t)lo->ref.nfpf * hi->ref.nfpf;
            }
        }
    }
    return P;
}

struct GroupLayout {
    size_t U, R1, R2, RES, UF0, UF1, FV, MET, NRM, MFLUX, PART, EINST, WALL;
};
struct Layout {
    GroupLayout g[frk::kMaxGroups];
    size_t BTAG, BVREF, STAGE, PROBES, PACC, PHIST, FORCE, PART_SUMS, RED, MORT, MATS, total;
};

Layout make_layout(const Plan &P, int n_inst, bool fp64, bool visc) {
    const size_t rs = fp64 ? 8 : 4;
    const int dim = P.dim, V = dim + 2, MS = dim * dim + 1;
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + std::max<size_t>(bytes, 16)); return at; };
    for (int g = 0; g < P.G; ++g) {
        const int n = P.degree[g] + 1;
        const int nsp = dim == 2 ? n * n : n * n * n, nfp = 2 * dim * (dim == 2 ? n : n * n);
        const int64_t E = P.E[g], box = P.box_lo[g] + P.box_hi[g];
        const size_t st = (size_t)E * nsp * V * rs, fc = ((size_t)E * nfp + box) * V * rs;
        GroupLayout &G = L.g[g];
        G.U = take(st);
        G.R1 = take(st);
        G.R2 = take(st);
        G.RES = take(st);
        G.UF0 = take(fc);
        G.UF1 = take(fc);
        G.FV = take(visc ? fc : 16);
        G.MET = take((size_t)E * nsp * MS * rs);
        G.NRM = take((size_t)E * nfp * dim * rs);
        G.MFLUX = take((size_t)box * V * rs);
        G.PART = take((size_t)E * nfp * 4);
        G.EINST = take((size_t)E * 4);
        G.WALL = take((size_t)P.n_wall[g] * 4);
    }
    L.BTAG = take((size_t)P.nb * 4);
    L.BVREF = take((size_t)P.nb * dim * rs);
    L.STAGE = take((size_t)P.stage_doubles * 8);
    L.PROBES = take(sizeof(frk::ProbeDesc) * kMaxProbes);
    L.PACC = take(sizeof(frk::ProbeAcc) * kMaxProbes);
    L.PHIST = take(sizeof(double) * kMaxProbes * frk::kHistLen);
    L.FORCE = take((size_t)n_inst * 3 * 8);
    L.PART_SUMS = take((size_t)frk::kMaxGroups * kPartialBlocks * (2 * V + 1) * 8);
    L.RED = take((size_t)(V + 1) * 8);
    L.MORT = take((size_t)P.n_mortar * sizeof(frk::MortarFace));
    L.MATS = take((size_t)P.mat_reals * rs);
    L.total = o;
    return L;
}

template <typename real>
void fill_args(const fr_solver *s, int g, frk::KArgs<real> &a) {
    const Group &G = s->grp[g];
    std::memset(&a, 0, sizeof(a));
    a.U = (real *)G.U;
    a.R1 = (real *)G.R1;
    a.R2 = (real *)G.R2;
    a.RES = (real *)G.RES;
    a.FV = (real *)G.FV;
    a.MET = (const real *)G.MET;
    a.NRM = (const real *)G.NRM;
    a.PART = G.PART;
    a.BTAG = s->BTAG;
    a.BVREF = (const real *)s->BVREF;
    a.EINST = G.EINST;
    a.fp_real = G.fp_real;
    a.fp_lo_end = G.fp_real + G.n_box_lo;
    a.MFLUX = (const real *)G.MFLUX;
    a.group = g;
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
    const RefElem &r = G.ref;
    for (int i = 0; i < G.N; ++i) {
        for (int mm = 0; mm < G.N; ++mm) a.opD1[i * frk::kMaxN + mm] = r.D1[i][mm];
        a.opL[i] = r.lend[0][i];
        a.opL[frk::kMaxN + i] = r.lend[1][i];
        a.opGL[i] = r.dgL[i];
        a.opGR[i] = r.dgR[i];
        a.opW[i] = r.w[i];
        for (int mm = 0; mm < G.N; ++mm)
            a.opDT[i * frk::kMaxN + mm] = r.D1[i][mm] - r.dgR[i] * r.lend[1][mm] - r.dgL[i] * r.lend[0][mm];
    }
}

// A launch description independent of the precision.
struct Launch {
    int kind = 0, g = 0;
    int64_t elem0 = 0, n_elem = 0;
    const int32_t *elist = nullptr;
    int mode = 0, force = 0, integral_src = 0;
    double rk_a = 0, rk_b = 0, rk_c = 0;
    const void *UFin = nullptr;
    void *UFout = nullptr;
    int64_t stage_off = 0;        // doubles into the FP64 staging buffer
    int64_t partial_slot = 0;     // first partial-sum block of the launch
    int64_t n_partials = 0;       // K_REDUCE: partial-sum blocks to reduce
    int grid = 1;
};

template <typename real>
cudaError_t do_launch(const fr_solver *s, const Launch &L) {
    frk::KArgs<real> a;
    fill_args(s, L.g, a);
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
    a.stage64 = s->stage64 + L.stage_off;
    a.stage64_out = s->stage64 + L.stage_off;
    a.partials = s->partials + L.partial_slot * (2 * s->V + 1);
    if (L.n_partials > 0) a.n_partials = L.n_partials;
    const int N = s->grp[L.g].N;
    const bool visc = s->visc;
    if constexpr (std::is_same<real, float>::value) {
        return s->dim == 2 ? frk::launch_2_f32(N, L.kind, visc, a, L.grid, s->stream)
                           : frk::launch_3_f32(N, L.kind, visc, a, L.grid, s->stream);
    } else {
        return s->dim == 2 ? frk::launch_2_f64(N, L.kind, visc, a, L.grid, s->stream)
                           : frk::launch_3_f64(N, L.kind, visc, a, L.grid, s->stream);
    }
}

template <typename real>
cudaError_t do_mortar(const fr_solver *s, int pass, int par, int64_t m0, int64_t count) {
    frk::MArgs<real> a;
    std::memset(&a, 0, sizeof(a));
    for (size_t g = 0; g < s->grp.size(); ++g) {
        const Group &G = s->grp[g];
        a.UF[g] = (real *)G.UF[par];
        a.FV[g] = (const real *)G.FV;
        a.NRM[g] = (const real *)G.NRM;
        a.MFLUX[g] = (real *)G.MFLUX;
        a.fp_real[g] = G.fp_real;
    }
    a.faces = s->MORT + m0;
    a.n_faces = count;
    a.mats = (const real *)s->MATS;
    a.gamma = (real)s->cfg.gamma;
    a.ldg_beta = (real)s->cfg.ldg_beta;
    a.ldg_tau = (real)s->cfg.ldg_tau;
    a.flux = s->cfg.flux;
    a.ldg = s->cfg.viscous_scheme == FR_VISC_LDG ? 1 : 0;
    a.visc = s->visc ? 1 : 0;
    a.pass = pass;
    if constexpr (std::is_same<real, float>::value)
        return s->dim == 2 ? frk::mortar_2_f32(a, s->stream) : frk::mortar_3_f32(a, s->stream);
    else
        return s->dim == 2 ? frk::mortar_2_f64(a, s->stream) : frk::mortar_3_f64(a, s->stream);
}

// profiling kinds of fr_profile_steps
enum ProfKind { P_FLUX = 0, P_GRAD = 1, P_PROBE = 2, P_FORCE = 3, P_OTHER = 4 };

int prof_kind(const Launch &L) {
    if (L.kind == frk::K_FLUX) return P_FLUX;
    if (L.kind == frk::K_GRAD) return L.force ? P_FORCE : P_GRAD;
    if (L.kind == frk::K_PROBE) return P_PROBE;
    return P_OTHER;
}

template <typename F>
cudaError_t timed(const fr_solver *s, int kind, F &&fn) {
    if (!s->profiling) return fn();
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    cudaEventRecord(a, s->stream);
    e = fn();
    cudaEventRecord(b, s->stream);
    const_cast<fr_solver *>(s)->prof.push_back({kind, {a, b}});
    return e;
}

cudaError_t launch(const fr_solver *s, const Launch &L) {
    return timed(s, prof_kind(L), [&] { return s->fp64 ? do_launch<double>(s, L) : do_launch<float>(s, L); });
}

// mortar pass over the faces [m0, m0 + count) on face buffer parity par
cudaError_t mortar(const fr_solver *s, int pass, int par, int64_t m0, int64_t count) {
    if (count <= 0) return cudaSuccess;
    return timed(s, P_OTHER, [&] {
        return s->fp64 ? do_mortar<double>(s, pass, par, m0, count) : do_mortar<float>(s, pass, par, m0, count);
    });
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
    const int G = (int)s->grp.size();
    for (int st = 0; st < stages; ++st) {
        if (s->visc) {
            for (int g = 0; g < G; ++g) {
                Launch l;
                l.kind = frk::K_GRAD;
                l.g = g;
                l.n_elem = s->grp[g].E;
                l.UFin = s->grp[g].UF[par];
                FR_CK(launch(s, l));
                ++cnt;
            }
        }
        if (s->n_mortar > 0) {
            FR_CK(mortar(s, 1, par, 0, s->n_mortar));
            ++cnt;
        }
        for (int g = 0; g < G; ++g) {
            Launch f;
            f.kind = frk::K_FLUX;
            f.g = g;
            f.n_elem = s->grp[g].E;
            f.UFin = s->grp[g].UF[par];
            f.UFout = s->grp[g].UF[par ^ 1];
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
        }
        if (s->n_mortar > 0) {
            FR_CK(mortar(s, 0, par ^ 1, 0, s->n_mortar));
            ++cnt;
        }
        par ^= 1;
    }
    for (int g = 0; g < G; ++g) {
        if (s->grp[g].n_probe <= 0) continue;
        Launch pr;
        pr.kind = frk::K_PROBE;
        pr.g = g;
        FR_CK(launch(s, pr));
        ++cnt;
    }
    for (int g = 0; g < G; ++g) {
        if (s->grp[g].n_wall <= 0) continue;
        Launch fo;
        fo.kind = frk::K_GRAD;
        fo.g = g;
        fo.force = 1;
        fo.elist = s->grp[g].WALL;
        fo.n_elem = s->grp[g].n_wall;
        fo.UFin = s->grp[g].UF[par];
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
    const int G = (int)s->grp.size();
    if (s->visc) {
        for (int g = 0; g < G; ++g) {
            Launch l;
            l.kind = frk::K_GRAD;
            l.g = g;
            l.elem0 = s->grp[g].off[inst];
            l.n_elem = s->grp[g].ne[inst];
            l.UFin = s->grp[g].UF[s->parity];
            FR_CK(launch(s, l));
        }
    }
    FR_CK(mortar(s, 1, s->parity, s->moff[inst], s->mcnt[inst]));
    for (int g = 0; g < G; ++g) {
        Launch f;
        f.kind = frk::K_FLUX;
        f.g = g;
        f.elem0 = s->grp[g].off[inst];
        f.n_elem = s->grp[g].ne[inst];
        f.UFin = s->grp[g].UF[s->parity];
        f.mode = mode;
        FR_CK(launch(s, f));
    }
    return FR_OK;
}

fr_status reduce_integral(fr_solver *s, int inst, int src, double *out_sums, double *out_bad) {
    const int G = (int)s->grp.size();
    // the partial-sum blocks are shared out among the degree groups, so the
    // ordered reduction reads kPartialBlocks slots whatever the number of groups
    const int per = std::max(1, kPartialBlocks / G);
    FR_CK(cudaMemsetAsync(s->partials, 0, (size_t)G * per * (2 * s->V + 1) * 8, s->stream));
    for (int g = 0; g < G; ++g) {
        if (s->grp[g].ne[inst] <= 0) continue;
        Launch in;
        in.kind = frk::K_INTEGRAL;
        in.g = g;
        in.elem0 = s->grp[g].off[inst];
        in.n_elem = s->grp[g].ne[inst];
        in.integral_src = src;
        in.partial_slot = (int64_t)g * per;
        in.grid = per;
        FR_CK(launch(s, in));
    }
    Launch rd;
    rd.kind = frk::K_REDUCE;
    rd.n_partials = (int64_t)G * per;
    FR_CK(launch(s, rd));
    std::vector<double> h(s->V + 1);
    FR_CK(cudaMemcpyAsync(h.data(), s->reduce_out, h.size() * 8, cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    for (int v = 0; v < s->V; ++v) out_sums[v] = h[v];
    if (out_bad) *out_bad = h[s->V];
    return FR_OK;
}

// instance spread over several groups?
bool spread(const fr_solver *s, int inst) { return !s->egroup[inst].empty(); }

// staging offset (doubles) of group g's block for one instance
int64_t stage_block(const fr_solver *s, int inst, int g) {
    int64_t o = 0;
    for (int h = 0; h < g; ++h) o += s->grp[h].ne[inst] * s->grp[h].nsp * s->V;
    return o;
}

}  // namespace
}  // namespace fr

using namespace fr;

extern "C" const char *fr_last_error(void) { return fr::g_last_error.c_str(); }

extern "C" size_t fr_workspace_bytes(fr_mesh *const *meshes, int n_inst, const fr_config *cfg) {
    if (check_batch(meshes, n_inst, cfg) != FR_OK) return 0;
    const Plan P = make_plan(meshes, n_inst);
    if (P.G > frk::kMaxGroups) return 0;
    return make_layout(P, n_inst, cfg->precision == FR_FP64, cfg->viscous != 0).total;
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
    fr::Range nvtx_range("fr_solver_create");
    if (!out) { set_error("null output pointer"); return FR_ERR_INVALID_ARG; }
    *out = nullptr;
    fr_status st = check_batch(meshes, n_inst, cfg);
    if (st != FR_OK) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        set_error("workspace must be a non-null device pointer aligned to 256 bytes");
        return FR_ERR_WORKSPACE;
    }
    const Plan P = make_plan(meshes, n_inst);
    auto s = std::make_unique<fr_solver>();
    const int dim = P.dim;
    s->dim = dim;
    s->n_inst = n_inst;
    s->cfg = *cfg;
    s->fp64 = cfg->precision == FR_FP64;
    s->visc = cfg->viscous != 0;
    s->V = dim + 2;
    s->MS = dim * dim + 1;
    s->rsz = s->fp64 ? 8 : 4;
    s->stream = (cudaStream_t)stream;
    s->nb = P.nb;
    s->n_mortar = P.n_mortar;
    s->grp.resize(P.G);
    for (int g = 0; g < P.G; ++g) {
        Group &G = s->grp[g];
        G.p = P.degree[g];
        G.N = G.p + 1;
        build_ref(G.ref, dim, G.p);
        G.nsp = G.ref.nsp;
        G.nfp = G.ref.nfp;
        G.nfpf = G.ref.nfpf;
        G.E = P.E[g];
        G.n_wall = P.n_wall[g];
        G.fp_real = G.E * G.nfp;
        G.n_box_lo = P.box_lo[g];
        G.n_box = P.box_lo[g] + P.box_hi[g];
        if (G.fp_real + G.n_box >= ((int64_t)1 << 31)) {
            set_error("batch too large for 32-bit flux-point indices");
            return FR_ERR_UNSUPPORTED;
        }
    }
    const Layout L = make_layout(P, n_inst, s->fp64, s->visc);
    if (ws_bytes < L.total) {
        set_error("workspace too small: need " + std::to_string(L.total) + " bytes");
        return FR_ERR_WORKSPACE;
    }
    char *w = (char *)workspace;
    for (int g = 0; g < P.G; ++g) {
        Group &G = s->grp[g];
        const GroupLayout &gl = L.g[g];
        G.U = w + gl.U; G.R1 = w + gl.R1; G.R2 = w + gl.R2; G.RES = w + gl.RES;
        G.UF[0] = w + gl.UF0; G.UF[1] = w + gl.UF1; G.FV = w + gl.FV;
        G.MET = w + gl.MET; G.NRM = w + gl.NRM; G.MFLUX = w + gl.MFLUX;
        G.PART = (int32_t *)(w + gl.PART); G.EINST = (int32_t *)(w + gl.EINST);
        G.WALL = (int32_t *)(w + gl.WALL);
    }
    s->BTAG = (int32_t *)(w + L.BTAG); s->BVREF = w + L.BVREF;
    s->stage64 = (double *)(w + L.STAGE);
    s->probes = (frk::ProbeDesc *)(w + L.PROBES);
    s->pacc = (frk::ProbeAcc *)(w + L.PACC);
    s->phist = (double *)(w + L.PHIST);
    s->force_acc = (double *)(w + L.FORCE);
    s->partials = (double *)(w + L.PART_SUMS);
    s->reduce_out = (double *)(w + L.RED);
    s->MORT = (frk::MortarFace *)(w + L.MORT);
    s->MATS = w + L.MATS;

    // element ranges of every instance in every group
    for (int g = 0; g < P.G; ++g) {
        s->grp[g].off.assign(n_inst, 0);
        s->grp[g].ne.assign(n_inst, 0);
    }
    {
        std::vector<int64_t> cursor(P.G, 0);
        for (int i = 0; i < n_inst; ++i)
            for (int g = 0; g < P.G; ++g) {
                s->grp[g].off[i] = cursor[g];
                for (const fr_mesh *pm : parts_of(meshes[i]))
                    if (P.group_of_degree[pm->p] == g) s->grp[g].ne[i] = pm->n_elem;
                cursor[g] += s->grp[g].ne[i];
            }
    }
    // host IO maps of instances spread over several groups
    s->egroup.resize(n_inst);
    s->elocal.resize(n_inst);
    s->esp.resize(n_inst);
    s->inst_nsp.assign(n_inst, 0);
    for (int i = 0; i < n_inst; ++i) {
        const fr_mesh *m = meshes[i];
        if (m->parts.empty()) {
            s->inst_nsp[i] = m->n_elem * m->ref.nsp;
            continue;
        }
        s->inst_nsp[i] = m->n_sp_total;
        s->egroup[i].resize(m->n_elem);
        s->elocal[i].resize(m->n_elem);
        s->esp[i].resize(m->n_elem);
        int64_t o = 0;
        for (int64_t e = 0; e < m->n_elem; ++e) {
            const fr_mesh *pm = m->parts[m->part_of[e]].get();
            s->egroup[i][e] = P.group_of_degree[pm->p];
            s->elocal[i][e] = m->local[e];
            s->esp[i][e] = o;
            o += pm->ref.nsp;
        }
    }

    // mortar faces, outbox rows and operators
    const int nfaces = 2 * dim;
    std::vector<std::vector<int64_t>> box_start(P.G);
    for (int g = 0; g < P.G; ++g) box_start[g].assign((size_t)s->grp[g].E * nfaces, -1);
    std::vector<frk::MortarFace> mfaces;
    s->moff.assign(n_inst, 0);
    s->mcnt.assign(n_inst, 0);
    {
        std::vector<int64_t> cur_lo(P.G, 0), cur_hi(P.G, 0);
        for (int i = 0; i < n_inst; ++i) {
            const fr_mesh *m = meshes[i];
            s->moff[i] = (int64_t)mfaces.size();
            for (const MortarLink &Lk : m->mortars) {
                const fr_mesh *lo = m->parts[Lk.part_lo].get(), *hi = m->parts[Lk.part_hi].get();
                const int glo = P.group_of_degree[lo->p], ghi = P.group_of_degree[hi->p];
                Group &Gl = s->grp[glo], &Gh = s->grp[ghi];
                const int64_t el = Gl.off[i] + Lk.e_lo, eh = Gh.off[i] + Lk.e_hi;
                frk::MortarFace F;
                F.glo = glo; F.ghi = ghi;
                F.nlo = Gl.nfpf; F.nhi = Gh.nfpf;
                F.lo_fp = el * Gl.nfp + (int64_t)Lk.f_lo * Gl.nfpf;
                F.hi_fp = eh * Gh.nfp + (int64_t)Lk.f_hi * Gh.nfpf;
                F.lo_box = Gl.fp_real + cur_lo[glo];
                F.hi_box = Gh.fp_real + Gh.n_box_lo + cur_hi[ghi];
                cur_lo[glo] += Gl.nfpf;
                cur_hi[ghi] += Gh.nfpf;
                F.mat = P.mat_off.at(mat_key(lo->p, hi->p, Lk.orient));
                box_start[glo][(size_t)el * nfaces + Lk.f_lo] = F.lo_box;
                box_start[ghi][(size_t)eh * nfaces + Lk.f_hi] = F.hi_box;
                mfaces.push_back(F);
            }
            s->mcnt[i] = (int64_t)mfaces.size() - s->moff[i];
        }
    }
    std::vector<double> mats((size_t)std::max<int64_t>(P.mat_reals, 1), 0.0);
    for (auto &kv : P.mat_off) {
        const int key = kv.first;
        const int plo = (key / 8) / 8, phi = (key / 8) % 8, orient = key % 8;
        RefElem rlo, rhi;
        build_ref(rlo, dim, plo);
        build_ref(rhi, dim, phi);
        std::vector<double> T, Pm;
        mortar_matrices(rlo, rhi, orient, T, Pm);
        std::copy(T.begin(), T.end(), mats.begin() + kv.second);
        std::copy(Pm.begin(), Pm.end(), mats.begin() + kv.second + (int64_t)T.size());
    }

    // host tables, FP64 first, cast once
    const int MS = s->MS;
    std::vector<double> bvref((size_t)std::max<int64_t>(P.nb, 1) * dim, 0.0);
    std::vector<int32_t> btag(std::max<int64_t>(P.nb, 1));
    std::vector<std::vector<double>> met(P.G), nrm(P.G);
    std::vector<std::vector<int32_t>> part(P.G), einst(P.G), wall(P.G);
    for (int g = 0; g < P.G; ++g) {
        const Group &G = s->grp[g];
        met[g].resize((size_t)G.E * G.nsp * MS);
        nrm[g].resize((size_t)G.E * G.nfp * dim);
        part[g].resize((size_t)G.E * G.nfp);
        einst[g].resize(G.E);
        wall[g].reserve(G.n_wall);
    }
    int64_t b = 0;
    for (int i = 0; i < n_inst; ++i) {
        for (const fr_mesh *m : parts_of(meshes[i])) {
            const int g = P.group_of_degree[m->p];
            const Group &G = s->grp[g];
            const int nsp = G.nsp, nfp = G.nfp;
            const int64_t off = G.off[i];
            for (int64_t e = 0; e < m->n_elem; ++e) {
                const int64_t ge = off + e;
                einst[g][ge] = i;
                for (int sp = 0; sp < nsp; ++sp) {
                    const size_t src = (size_t)e * nsp + sp;
                    for (int kk = 0; kk < dim * dim; ++kk)
                        met[g][((size_t)ge * nsp + sp) * MS + kk] = m->S[src * dim * dim + kk];
                    met[g][((size_t)ge * nsp + sp) * MS + dim * dim] = 1.0 / m->J[src];
                }
                bool has_wall = false;
                for (int f = 0; f < nfp; ++f) {
                    const size_t lf = (size_t)e * nfp + f;
                    for (int d = 0; d < dim; ++d) nrm[g][((size_t)ge * nfp + f) * dim + d] = m->nrm[lf * dim + d];
                    const int64_t pt = m->partner[lf];
                    const int32_t tag = m->bctag[lf];
                    if (pt >= 0) {
                        part[g][(size_t)ge * nfp + f] = (int32_t)(off * nfp + pt);
                    } else if (tag == kTagMortar) {
                        const int64_t b0 = box_start[g][(size_t)ge * nfaces + f / G.nfpf];
                        if (b0 < G.fp_real || b0 + G.nfpf > G.fp_real + G.n_box) {
                            set_error("face joining two degrees without its mortar record");
                            return FR_ERR_MESH;
                        }
                        part[g][(size_t)ge * nfp + f] = (int32_t)(b0 + f % G.nfpf);
                    } else {
                        part[g][(size_t)ge * nfp + f] = (int32_t)(-1 - b);
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
                if (has_wall) wall[g].push_back((int32_t)ge);
            }
        }
        // slim host copy for probe location
        const fr_mesh *m = meshes[i];
        auto hm = std::make_unique<fr_mesh>();
        hm->dim = m->dim; hm->p = m->p; hm->q = m->q; hm->ref = m->ref; hm->n_elem = m->n_elem;
        hm->nodes = m->nodes;
        s->host_meshes.push_back(std::move(hm));
    }
    std::vector<char> tmp;
    cudaStream_t cs = s->stream;
    auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(cs);
    };
    auto up_real = [&](void *dst, const std::vector<double> &src, size_t n) -> cudaError_t {
        if (s->fp64) return up(dst, src.data(), n * 8);
        to_real<float>(tmp, src);
        return up(dst, tmp.data(), n * 4);
    };
    for (int g = 0; g < P.G; ++g) {
        Group &G = s->grp[g];
        FR_CK(up_real(G.MET, met[g], met[g].size()));
        FR_CK(up_real(G.NRM, nrm[g], nrm[g].size()));
        FR_CK(up(G.PART, part[g].data(), part[g].size() * 4));
        FR_CK(up(G.EINST, einst[g].data(), einst[g].size() * 4));
        FR_CK(up(G.WALL, wall[g].data(), wall[g].size() * 4));
        const size_t st_bytes = (size_t)G.E * G.nsp * s->V * s->rsz;
        const size_t fc_bytes = ((size_t)G.E * G.nfp + G.n_box) * s->V * s->rsz;
        FR_CK(cudaMemsetAsync(G.U, 0, st_bytes, cs));
        FR_CK(cudaMemsetAsync(G.R1, 0, st_bytes, cs));
        FR_CK(cudaMemsetAsync(G.R2, 0, st_bytes, cs));
        FR_CK(cudaMemsetAsync(G.RES, 0, st_bytes, cs));
        FR_CK(cudaMemsetAsync(G.UF[0], 0, fc_bytes, cs));
        FR_CK(cudaMemsetAsync(G.UF[1], 0, fc_bytes, cs));
        if (s->visc) FR_CK(cudaMemsetAsync(G.FV, 0, fc_bytes, cs));
        FR_CK(cudaMemsetAsync(G.MFLUX, 0, (size_t)G.n_box * s->V * s->rsz, cs));
    }
    FR_CK(up_real(s->BVREF, bvref, (size_t)P.nb * dim));
    FR_CK(up(s->BTAG, btag.data(), (size_t)P.nb * 4));
    FR_CK(up(s->MORT, mfaces.data(), mfaces.size() * sizeof(frk::MortarFace)));
    FR_CK(up_real(s->MATS, mats, (size_t)P.mat_reals));
    FR_CK(cudaMemsetAsync(s->pacc, 0, sizeof(frk::ProbeAcc) * kMaxProbes, cs));
    FR_CK(cudaMemsetAsync(s->force_acc, 0, (size_t)n_inst * 3 * 8, cs));
    FR_CK(cudaStreamSynchronize(cs));
    for (int g = 0; g < P.G; ++g) {
        const int N = s->grp[g].N;
        cudaError_t pe;
        if (dim == 2) pe = s->fp64 ? frk::prepare_2_f64(N, s->visc) : frk::prepare_2_f32(N, s->visc);
        else pe = s->fp64 ? frk::prepare_3_f64(N, s->visc) : frk::prepare_3_f32(N, s->visc);
        FR_CK(pe);
    }
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

namespace {

// Enqueue the upload of one instance's FP64 host state (the ABI's element
// order) and the derivation of its face values; no synchronisation.  An
// instance spread over several degree groups is reordered on the host into
// `tmp`, which must stay alive until the stream has been synchronised.
fr_status enqueue_upload(fr_solver *s, int inst, const double *u, std::vector<double> &tmp) {
    const int V = s->V;
    const size_t n = (size_t)s->inst_nsp[inst] * V;
    if (!spread(s, inst)) {
        FR_CK(cudaMemcpyAsync(s->stage64, u, n * 8, cudaMemcpyHostToDevice, s->stream));
    } else {
        // host reorder: element order -> group blocks
        tmp.resize(n);
        std::vector<int64_t> blk(s->grp.size());
        for (size_t g = 0; g < s->grp.size(); ++g) blk[g] = stage_block(s, inst, (int)g);
        for (size_t e = 0; e < s->egroup[inst].size(); ++e) {
            const int g = s->egroup[inst][e];
            const size_t cnt = (size_t)s->grp[g].nsp * V;
            std::memcpy(&tmp[blk[g] + s->elocal[inst][e] * cnt], u + s->esp[inst][e] * V, cnt * 8);
        }
        FR_CK(cudaMemcpyAsync(s->stage64, tmp.data(), n * 8, cudaMemcpyHostToDevice, s->stream));
    }
    for (size_t g = 0; g < s->grp.size(); ++g) {
        const Group &G = s->grp[g];
        if (G.ne[inst] <= 0) continue;
        Launch c;
        c.kind = frk::K_TO_REAL;
        c.g = (int)g;
        c.elem0 = G.off[inst];
        c.n_elem = G.ne[inst];
        c.stage_off = stage_block(s, inst, (int)g);
        c.grid = grid_for(G.ne[inst] * G.nsp * V);
        FR_CK(launch(s, c));
        Launch in;
        in.kind = frk::K_INTERP;
        in.g = (int)g;
        in.elem0 = G.off[inst];
        in.n_elem = G.ne[inst];
        in.UFout = G.UF[s->parity];
        FR_CK(launch(s, in));
    }
    FR_CK(mortar(s, 0, s->parity, s->moff[inst], s->mcnt[inst]));
    return FR_OK;
}

// Enqueue the FP64 conversion of one instance's state (src 0) or residual
// (src 1) and its download to u; no synchronisation.  An instance spread over
// several degree groups lands in `tmp` and is put in element order by
// finish_download once the stream has been synchronised.
fr_status enqueue_download(fr_solver *s, int inst, int src, double *u, std::vector<double> &tmp) {
    const int V = s->V;
    const size_t n = (size_t)s->inst_nsp[inst] * V;
    for (size_t g = 0; g < s->grp.size(); ++g) {
        const Group &G = s->grp[g];
        if (G.ne[inst] <= 0) continue;
        Launch c;
        c.kind = frk::K_TO_F64;
        c.g = (int)g;
        c.elem0 = G.off[inst];
        c.n_elem = G.ne[inst];
        c.integral_src = src;
        c.stage_off = stage_block(s, inst, (int)g);
        c.grid = grid_for(G.ne[inst] * G.nsp * V);
        FR_CK(launch(s, c));
    }
    if (!spread(s, inst)) {
        FR_CK(cudaMemcpyAsync(u, s->stage64, n * 8, cudaMemcpyDeviceToHost, s->stream));
    } else {
        tmp.resize(n);
        FR_CK(cudaMemcpyAsync(tmp.data(), s->stage64, n * 8, cudaMemcpyDeviceToHost, s->stream));
    }
    return FR_OK;
}

void finish_download(const fr_solver *s, int inst, const std::vector<double> &tmp, double *u) {
    if (!spread(s, inst)) return;
    const int V = s->V;
    std::vector<int64_t> blk(s->grp.size());
    for (size_t g = 0; g < s->grp.size(); ++g) blk[g] = stage_block(s, inst, (int)g);
    for (size_t e = 0; e < s->egroup[inst].size(); ++e) {
        const int g = s->egroup[inst][e];
        const size_t cnt = (size_t)s->grp[g].nsp * V;
        std::memcpy(u + s->esp[inst][e] * V, &tmp[blk[g] + s->elocal[inst][e] * cnt], cnt * 8);
    }
}

}  // namespace

extern "C" fr_status fr_set_state(fr_solver *s, int inst, const double *u) {
    fr::Range nvtx_range("fr_set_state");
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!u) { set_error("null state"); return FR_ERR_INVALID_ARG; }
    std::vector<double> tmp;
    st = enqueue_upload(s, inst, u, tmp);
    if (st != FR_OK) return st;
    FR_CK(cudaStreamSynchronize(s->stream));
    return FR_OK;
}

static fr_status copy_out(fr_solver *s, int inst, int src, double *u) {
    std::vector<double> tmp;
    fr_status st = enqueue_download(s, inst, src, u, tmp);
    if (st != FR_OK) return st;
    FR_CK(cudaStreamSynchronize(s->stream));
    finish_download(s, inst, tmp, u);
    return FR_OK;
}

extern "C" fr_status fr_set_states(fr_solver *s, const double *u) {
    fr::Range nvtx_range("fr_set_states");
    if (!s || !u) { set_error("null argument"); return FR_ERR_INVALID_ARG; }
    std::vector<std::vector<double>> tmp(s->n_inst);
    size_t off = 0;
    for (int i = 0; i < s->n_inst; ++i) {
        fr_status st = enqueue_upload(s, i, u + off, tmp[i]);
        if (st != FR_OK) {
            cudaStreamSynchronize(s->stream);   // the host buffers above must outlive the copies
            return st;
        }
        off += (size_t)s->inst_nsp[i] * s->V;
    }
    FR_CK(cudaStreamSynchronize(s->stream));
    return FR_OK;
}

extern "C" fr_status fr_get_states(fr_solver *s, double *u) {
    fr::Range nvtx_range("fr_get_states");
    if (!s || !u) { set_error("null argument"); return FR_ERR_INVALID_ARG; }
    std::vector<std::vector<double>> tmp(s->n_inst);
    std::vector<size_t> off(s->n_inst + 1, 0);
    for (int i = 0; i < s->n_inst; ++i) off[i + 1] = off[i] + (size_t)s->inst_nsp[i] * s->V;
    for (int i = 0; i < s->n_inst; ++i) {
        fr_status st = enqueue_download(s, i, 0, u + off[i], tmp[i]);
        if (st != FR_OK) {
            cudaStreamSynchronize(s->stream);
            return st;
        }
    }
    FR_CK(cudaStreamSynchronize(s->stream));
    for (int i = 0; i < s->n_inst; ++i) finish_download(s, i, tmp[i], u + off[i]);
    return FR_OK;
}

extern "C" fr_status fr_get_state(fr_solver *s, int inst, double *u) {
    fr::Range nvtx_range("fr_get_state");
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!u) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    return copy_out(s, inst, 0, u);
}

extern "C" fr_status fr_residual(fr_solver *s, int inst, double *r) {
    fr::Range nvtx_range("fr_residual");
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!r) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    st = residual_into_res(s, inst, frk::M_RESIDUAL);
    if (st != FR_OK) return st;
    return copy_out(s, inst, 1, r);
}

extern "C" fr_status fr_rk_step(fr_solver *s, int n_steps) {
    fr::Range nvtx_range("fr_rk_step");
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
    fr::Range nvtx_range("fr_profile_steps");
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
    // the element's degree group and index there
    int g = 0;
    int64_t le = e;
    if (spread(s, inst)) {
        g = s->egroup[inst][e];
        le = s->elocal[inst][e];
    } else {
        for (size_t h = 0; h < s->grp.size(); ++h)
            if (s->grp[h].ne[inst] > 0) g = (int)h;
    }
    frk::ProbeDesc d;
    std::memset(&d, 0, sizeof(d));
    d.elem = s->grp[g].off[inst] + le;
    d.inst = inst;
    d.group = g;
    ref_interp(s->grp[g].ref, xi, d.w);
    const int id = s->n_probe;
    FR_CK(cudaMemcpyAsync(&s->probes[id], &d, sizeof(d), cudaMemcpyHostToDevice, s->stream));
    FR_CK(cudaMemsetAsync(&s->pacc[id], 0, sizeof(frk::ProbeAcc), s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    s->n_probe += 1;
    s->grp[g].n_probe += 1;
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

// Accumulator checkpoint: [steps in the window, number of probes, wall-force
// sums n_inst x 3, probe accumulators n_probe x 16, sample rings n_probe x kHistLen]
extern "C" int64_t fr_accumulators_size(const fr_solver *s) {
    if (!s) return -1;
    return 2 + (int64_t)s->n_inst * 3 + (int64_t)s->n_probe * (int64_t)(sizeof(frk::ProbeAcc) / 8) +
           (int64_t)s->n_probe * frk::kHistLen;
}

extern "C" fr_status fr_get_accumulators(fr_solver *s, double *out) {
    if (!s || !out) { set_error("null argument"); return FR_ERR_INVALID_ARG; }
    const size_t na = sizeof(frk::ProbeAcc) / 8;
    out[0] = (double)s->steps_since_reset;
    out[1] = (double)s->n_probe;
    double *f = out + 2, *pa = f + (size_t)s->n_inst * 3, *ph = pa + (size_t)s->n_probe * na;
    FR_CK(cudaMemcpyAsync(f, s->force_acc, (size_t)s->n_inst * 3 * 8, cudaMemcpyDeviceToHost, s->stream));
    if (s->n_probe > 0) {
        FR_CK(cudaMemcpyAsync(pa, s->pacc, (size_t)s->n_probe * sizeof(frk::ProbeAcc), cudaMemcpyDeviceToHost,
                              s->stream));
        FR_CK(cudaMemcpyAsync(ph, s->phist, (size_t)s->n_probe * frk::kHistLen * 8, cudaMemcpyDeviceToHost,
                              s->stream));
    }
    FR_CK(cudaStreamSynchronize(s->stream));
    return FR_OK;
}

extern "C" fr_status fr_set_accumulators(fr_solver *s, const double *in) {
    if (!s || !in) { set_error("null argument"); return FR_ERR_INVALID_ARG; }
    if (in[1] != (double)s->n_probe || !(in[0] >= 0.0)) {
        set_error("accumulator checkpoint is for " + std::to_string((int64_t)in[1]) + " probes, the solver has " +
                  std::to_string(s->n_probe));
        return FR_ERR_INVALID_ARG;
    }
    const size_t na = sizeof(frk::ProbeAcc) / 8;
    const double *f = in + 2, *pa = f + (size_t)s->n_inst * 3, *ph = pa + (size_t)s->n_probe * na;
    FR_CK(cudaMemcpyAsync(s->force_acc, f, (size_t)s->n_inst * 3 * 8, cudaMemcpyHostToDevice, s->stream));
    if (s->n_probe > 0) {
        FR_CK(cudaMemcpyAsync(s->pacc, pa, (size_t)s->n_probe * sizeof(frk::ProbeAcc), cudaMemcpyHostToDevice,
                              s->stream));
        FR_CK(cudaMemcpyAsync(s->phist, ph, (size_t)s->n_probe * frk::kHistLen * 8, cudaMemcpyHostToDevice,
                              s->stream));
    }
    FR_CK(cudaStreamSynchronize(s->stream));
    s->steps_since_reset = (int64_t)in[0];
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
    fr::Range nvtx_range("fr_conservation");
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!sums) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    st = residual_into_res(s, inst, frk::M_RESIDUAL_J);
    if (st != FR_OK) return st;
    return reduce_integral(s, inst, 1, sums, nullptr);
}

extern "C" fr_status fr_integral(fr_solver *s, int inst, double *sums, int64_t *n_nonfinite) {
    fr::Range nvtx_range("fr_integral");
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

// K_INTEGRAL of one group's part of an instance into the blocks
// [block0, block0 + grid) of the scratch array, or (kind K_REDUCE) the
// reduction of the first ``grid`` blocks
template <typename real>
cudaError_t launch_static(const fr_solver *s, int kind, int g, int inst, int64_t block0, int grid,
                          double *scratch) {
    frk::KArgs<real> a;
    fill_args(s, g, a);
    a.elem0 = s->grp[g].off[inst];
    a.n_elem = s->grp[g].ne[inst];
    a.integral_src = 0;
    a.partials = scratch + block0 * (2 * s->V + 1);   // the kernels' slot stride
    a.n_partials = grid;
    a.reduce_out = scratch + (size_t)kStaticBlocks * kStaticSlotsPerBlock;
    const int N = s->grp[g].N;
    if constexpr (std::is_same<real, float>::value) {
        return s->dim == 2 ? frk::launch_2_f32(N, kind, s->visc, a, grid, s->stream)
                           : frk::launch_3_f32(N, kind, s->visc, a, grid, s->stream);
    } else {
        return s->dim == 2 ? frk::launch_2_f64(N, kind, s->visc, a, grid, s->stream)
                           : frk::launch_3_f64(N, kind, s->visc, a, grid, s->stream);
    }
}

}  // namespace
}  // namespace fr

extern "C" fr_status fr_integral_static(fr_solver *s, int inst, double *sums, int64_t *n_nonfinite) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!sums) { set_error("null output"); return FR_ERR_INVALID_ARG; }
    const int per_block = fr::kStaticThreads * fr::kStaticItemsPerThread;
    // blocks per degree group: each group's points are summed by its own blocks
    const int G = (int)s->grp.size();
    std::vector<int> grids(G, 0);
    int64_t items = 0, blocks = 0;
    for (int g = 0; g < G; ++g) {
        const int64_t it = s->grp[g].ne[inst] * (int64_t)s->grp[g].nsp;
        items += it;
        grids[g] = it > 0 ? (int)((it + per_block - 1) / per_block) : 0;
        blocks += grids[g];
    }
    if (items > fr::kStaticMaxItems || blocks > fr::kStaticBlocks) {
        set_error("fr_integral_static: instance has " + std::to_string(items) +
                  " solution points, more than the static scratch serves (" +
                  std::to_string(fr::kStaticMaxItems) + "); use fr_integral");
        return FR_ERR_INVALID_ARG;
    }
    double *scratch = nullptr;
    st = fr::static_scratch(&scratch);
    if (st != FR_OK) return st;
    // every block writes all of its slots; the result slots are cleared anyway
    FR_CK(cudaMemsetAsync(scratch, 0, fr::kStaticDoubles * sizeof(double), s->stream));
    int64_t b0 = 0;
    for (int g = 0; g < G; ++g) {
        if (grids[g] == 0) continue;
        FR_CK(s->fp64 ? fr::launch_static<double>(s, frk::K_INTEGRAL, g, inst, b0, grids[g], scratch)
                      : fr::launch_static<float>(s, frk::K_INTEGRAL, g, inst, b0, grids[g], scratch));
        b0 += grids[g];
    }
    const int nb = (int)std::max<int64_t>(b0, 1);
    FR_CK(s->fp64 ? fr::launch_static<double>(s, frk::K_REDUCE, 0, inst, 0, nb, scratch)
                  : fr::launch_static<float>(s, frk::K_REDUCE, 0, inst, 0, nb, scratch));
    double h[6] = {0, 0, 0, 0, 0, 0};
    FR_CK(cudaMemcpyAsync(h, scratch + (size_t)fr::kStaticBlocks * fr::kStaticSlotsPerBlock,
                          (size_t)(s->V + 1) * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    for (int v = 0; v < s->V; ++v) sums[v] = h[v];
    if (n_nonfinite) *n_nonfinite = (int64_t)h[s->V];
    if (h[s->V] > 0) { set_error("non-finite values in the state"); return FR_ERR_NONFINITE; }
    return FR_OK;
}
