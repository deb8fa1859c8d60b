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
#include <cstdlib>
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
    char *FV = nullptr, *MET = nullptr, *NRM = nullptr, *MFLUX = nullptr, *DIVREF = nullptr;
    // fused viscous stage: second (ping-pong) buffer of the inbound gradient
    // flux parts (the first is FV) and the partner lifting coefficients
    char *FV2 = nullptr, *LFP = nullptr;
    // adaptive steps: third RK register (u_n) and the group's first element
    // in the batch's per-element error array
    char *R3 = nullptr;
    int64_t ebase = 0;
    int32_t *PART = nullptr, *EINST = nullptr, *WALL = nullptr;
    bool use_divref = false;   // FP32: the reference flux has a residual here
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
    // FP32: reference state of the perturbation storage (FP32 constants of the
    // kernels, the FP64 conserved values and pressure, the FP64 reference flux)
    frk::RefState<float> ref32{};
    double uref64[5] = {0, 0, 0, 0, 0}, pref64 = 0.0;
    double vref64[3] = {0, 0, 0};
    double Fref[3][5] = {};
    // FP32: sum over each instance's wall points of w n (FP64, host); the
    // kernels accumulate w ((p - p_r) n - tau n) and fr_forces adds p_r times it
    std::vector<double> wall_nsum;
    frk::ProbeDesc *probes = nullptr;
    frk::ProbeAcc *pacc = nullptr;
    double *phist = nullptr;
    int n_probe = 0;
    std::vector<int> probe_inst;
    std::vector<int64_t> probe_elem;   // element (within its degree group) of each observer
    int parity = 0;
    int64_t steps_since_reset = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t launches_per_step = 0, last_launches = 0;
    // non-finite scan every check_every steps (cfg.check_every; 0: off)
    int32_t *FLAGS = nullptr;
    int64_t steps_since_check = 0;
    // BR2 stages as one fused kernel (K_STAGE) instead of K_GRAD + K_FLUX
    bool fused = false;
    // FP32: fluxes about element-local references (cfg.flux_reference 0) or the free stream
    bool local_ref = true;
    // register level of the stage kernels (fr_tune)
    int regs_level = 0;
    // FP32: line contractions on the tensor cores (3xTF32 mma.sync; fr_tune)
    bool tc = false;
    // adaptive steps (FR_BS32): step-control records [n_inst][kAdStride],
    // accepted flags, per-element error sums, instance ranges of those; the
    // stage-1 evaluation of fresh instances is pending (bs_start)
    bool adapt = false, bs_start = false;
    double *ADAPT = nullptr, *ERRE = nullptr;
    int32_t *ACC = nullptr;
    frk::AdaptRange *ARANGE = nullptr;
    std::vector<double> adapt_init;   // host: the initial record of every instance
    // batch transfers: an auxiliary stream for the host-link copies (so that
    // one chunk's copy overlaps the previous chunk's conversion) and events
    cudaStream_t xfer = nullptr;
    cudaEvent_t xev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    std::string schedule_source = "default";
    double schedule_ms = 0.0;
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

// propagate a failed fr_status
#define FR_TRY(call)                      \
    do {                                  \
        const fr_status _st = (call);     \
        if (_st != FR_OK) return _st;     \
    } while (0)

// adaptive steps: end time and step cap (<= 0 in the configuration: none)
double eff_t_end(const fr_config &c) { return c.t_end > 0.0 ? c.t_end : INFINITY; }
double eff_dt_max(const fr_config &c) { return c.dt_max > 0.0 ? c.dt_max : INFINITY; }
// the first attempt's step from t = 0 (the rule of K_BS_CONTROL)
double first_step(const fr_config &c) {
    double h = std::min(c.dt, eff_dt_max(c));
    if (0.0 + h > eff_t_end(c)) h = eff_t_end(c) - 0.0;
    return std::max(h, 0.0);
}

fr_status check_batch(fr_mesh *const *meshes, int n_inst, const fr_config *cfg) {
    if (!meshes || n_inst <= 0 || !cfg) { set_error("invalid solver arguments"); return FR_ERR_INVALID_ARG; }
    for (int i = 0; i < n_inst; ++i) {
        if (!meshes[i]) { set_error("null mesh in batch"); return FR_ERR_INVALID_ARG; }
        if (meshes[i]->dim != meshes[0]->dim) {
            set_error("all meshes of a batch must share the dimension");
            return FR_ERR_UNSUPPORTED;
        }
    }
    if (cfg->rk != FR_RK4 && cfg->rk != FR_LSRK45 && cfg->rk != FR_BS32) { set_error("unknown rk scheme"); return FR_ERR_INVALID_ARG; }
    if (cfg->rk == FR_BS32) {
        const int V = meshes[0]->dim + 2;
        bool ok = cfg->dt > 0.0 && cfg->rtol >= 0.0;
        for (int v = 0; v < V; ++v) ok = ok && cfg->atol[v] >= 0.0 && cfg->atol[v] + cfg->rtol > 0.0;
        if (!ok) {
            set_error("adaptive steps need dt > 0, rtol >= 0 and atol_v >= 0 with atol_v + rtol > 0");
            return FR_ERR_INVALID_ARG;
        }
    }
    if (cfg->check_every < 0) { set_error("check_every must be >= 0"); return FR_ERR_INVALID_ARG; }
    if (cfg->flux_reference != 0 && cfg->flux_reference != 1) { set_error("unknown flux reference"); return FR_ERR_INVALID_ARG; }
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
        P.stage_doubles += nsp_inst * V;   // FP64 staging of the whole batch
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
    size_t U, R1, R2, RES, UF0, UF1, FV, MET, NRM, MFLUX, PART, EINST, WALL, DIVREF, FV2, LFP, R3;
};
struct Layout {
    GroupLayout g[frk::kMaxGroups];
    size_t BTAG, BVREF, STAGE, PROBES, PACC, PHIST, FORCE, PART_SUMS, RED, MORT, MATS, FLAGS;
    size_t ERRE, ADAPT, ACC, ARANGE, total;
};

Layout make_layout(const Plan &P, int n_inst, bool fp64, bool visc, bool adapt) {
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
        G.DIVREF = take(fp64 ? 16 : st);
        G.FV2 = take(visc ? fc : 16);
        G.LFP = take(visc ? (size_t)E * nfp * dim * rs : 16);
        G.R3 = take(adapt ? st : 16);
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
    L.FLAGS = take((size_t)n_inst * 4);
    int64_t e_all = 0;
    for (int g = 0; g < P.G; ++g) e_all += P.E[g];
    L.ERRE = take(adapt ? (size_t)e_all * 8 : 16);
    L.ADAPT = take((size_t)n_inst * frk::kAdStride * 8);
    L.ACC = take((size_t)n_inst * 4);
    L.ARANGE = take((size_t)n_inst * sizeof(frk::AdaptRange));
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
    a.gamma64 = s->cfg.gamma;
    a.pref64 = s->pref64;
    for (int v = 0; v < 5; ++v) a.uref64[v] = s->uref64[v];
    if constexpr (std::is_same<real, float>::value) a.ref = s->ref32;
    a.DIVREF = G.use_divref ? (const real *)G.DIVREF : nullptr;
    a.FLAGS = s->FLAGS;
    a.LFP = (const real *)G.LFP;
    a.local_ref = s->local_ref ? 1 : 0;
    a.regs_level = s->regs_level;
    a.tc = (s->tc && !s->fp64) ? 1 : 0;
    if (s->adapt) {
        a.ADAPT = s->ADAPT;
        a.ACC = s->ACC;
        a.R3 = (real *)G.R3;
        a.ERRE = s->ERRE + G.ebase;
        a.ARANGE = s->ARANGE;
        a.bs_rtol = (real)s->cfg.rtol;
        for (int v = 0; v < s->V; ++v) a.bs_atol[v] = (real)s->cfg.atol[v];
        a.t_end = eff_t_end(s->cfg);
        a.dt_max = eff_dt_max(s->cfg);
    }
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
    const void *FVin = nullptr;   // fused stage: inbound / outbound gradient flux parts
    void *FVout = nullptr;
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
    a.FVin = (const real *)L.FVin;
    a.FVout = (real *)L.FVout;
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
    if constexpr (std::is_same<real, float>::value) a.ref = s->ref32;
    if constexpr (std::is_same<real, float>::value)
        return s->dim == 2 ? frk::mortar_2_f32(a, s->stream) : frk::mortar_3_f32(a, s->stream);
    else
        return s->dim == 2 ? frk::mortar_2_f64(a, s->stream) : frk::mortar_3_f64(a, s->stream);
}

// profiling kinds of fr_profile_steps
enum ProfKind { P_FLUX = 0, P_GRAD = 1, P_PROBE = 2, P_FORCE = 3, P_OTHER = 4 };

int prof_kind(const Launch &L) {
    if (L.kind == frk::K_FLUX || L.kind == frk::K_STAGE) return P_FLUX;
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

// inbound gradient-flux-part buffer of face parity par (fused stage)
char *fvbuf(const Group &G, int par) { return par == 0 ? G.FV : G.FV2; }

// One stage evaluation reading face-buffer parity par (and writing par ^ 1):
// [gradient kernels,] mortar common fluxes, stage kernels with RK mode
// `mode`, mortar traces of the new state (not for M_BS_START and M_BS_4,
// which leave the state and the face buffers as they are).
fr_status enqueue_eval(fr_solver *s, int par, int mode, double rk_a, double rk_b, double rk_c, int64_t &cnt) {
    const int G = (int)s->grp.size();
    if (s->visc && !s->fused) {
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
        f.kind = s->fused ? frk::K_STAGE : frk::K_FLUX;
        f.g = g;
        f.n_elem = s->grp[g].E;
        f.UFin = s->grp[g].UF[par];
        f.UFout = s->grp[g].UF[par ^ 1];
        f.FVin = fvbuf(s->grp[g], par);
        f.FVout = fvbuf(s->grp[g], par ^ 1);
        f.mode = mode;
        f.rk_a = rk_a;
        f.rk_b = rk_b;
        f.rk_c = rk_c;
        FR_CK(launch(s, f));
        ++cnt;
    }
    if (s->n_mortar > 0 && mode != frk::M_BS_START && mode != frk::M_BS_4) {
        FR_CK(mortar(s, 0, par ^ 1, 0, s->n_mortar));
        ++cnt;
    }
    return FR_OK;
}

// Observers and wall forces after a step (face-buffer parity par holds the
// faces of the step's final state).
fr_status enqueue_samples(fr_solver *s, int par, int64_t &cnt) {
    const int G = (int)s->grp.size();
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
    return FR_OK;
}

// Face-buffer parity flips of one step (one per stage evaluation).
int step_flips(const fr_solver *s) {
    return s->cfg.rk == FR_RK4 ? 4 : s->cfg.rk == FR_LSRK45 ? 5 : 3;
}

// Face states (and, fused BR2, gradient flux parts) of the current state U
// of every instance into face-buffer parity par, mortar traces included.
fr_status enqueue_faces(fr_solver *s, int par, int64_t &cnt) {
    for (size_t g = 0; g < s->grp.size(); ++g) {
        const Group &G = s->grp[g];
        Launch in;
        in.kind = s->fused ? frk::K_INTERP_VISC : frk::K_INTERP;
        in.g = (int)g;
        in.n_elem = G.E;
        in.UFout = G.UF[par];
        in.FVout = fvbuf(G, par);
        FR_CK(launch(s, in));
        ++cnt;
    }
    if (s->n_mortar > 0) {
        FR_CK(mortar(s, 0, par, 0, s->n_mortar));
        ++cnt;
    }
    return FR_OK;
}

// One adaptive attempt (FR_BS32) from face-buffer parity p0: accept or roll
// back the previous attempt and form the first stage state (K_BS_COMMIT), its
// faces, the three stage evaluations (the last one computes k4 and writes no
// faces), the per-element errors, the controller, then the samples of
// accepted steps (on the faces of u_n+1, which the last evaluation read).
fr_status enqueue_attempt(fr_solver *s, int p0, int64_t *n_launch) {
    int par = p0;
    int64_t cnt = 0;
    for (size_t g = 0; g < s->grp.size(); ++g) {
        const Group &G = s->grp[g];
        Launch c;
        c.kind = frk::K_BS_COMMIT;
        c.g = (int)g;
        c.n_elem = G.E;
        c.grid = grid_for(G.E * G.nsp * s->V);
        FR_CK(launch(s, c));
        ++cnt;
    }
    FR_TRY(enqueue_faces(s, par, cnt));
    const int modes[3] = {frk::M_BS_2, frk::M_BS_3, frk::M_BS_4};
    for (int st = 0; st < 3; ++st) {
        FR_TRY(enqueue_eval(s, par, modes[st], 0.0, 0.0, 0.0, cnt));
        par ^= 1;
    }
    for (size_t g = 0; g < s->grp.size(); ++g) {
        Launch er;
        er.kind = frk::K_BS_ERROR;
        er.g = (int)g;
        er.n_elem = s->grp[g].E;
        FR_CK(launch(s, er));
        ++cnt;
    }
    Launch ct;
    ct.kind = frk::K_BS_CONTROL;
    ct.g = 0;
    ct.grid = s->n_inst;
    FR_CK(launch(s, ct));
    ++cnt;
    FR_TRY(enqueue_samples(s, par ^ 1, cnt));
    *n_launch = cnt;
    return FR_OK;
}

// Adaptive steps, after the last attempt of a call: U back to u_n where the
// last attempt was rejected, and the face data of every instance's current
// solution into face-buffer parity s->parity (the last stage evaluation of an
// attempt writes none), so that residuals, integrals and downloads between
// calls see the solution.
fr_status bs_settle(fr_solver *s, int64_t &cnt) {
    for (size_t g = 0; g < s->grp.size(); ++g) {
        const Group &G = s->grp[g];
        Launch c;
        c.kind = frk::K_BS_COMMIT;
        c.mode = 1;
        c.g = (int)g;
        c.n_elem = G.E;
        c.grid = grid_for(G.E * G.nsp * s->V);
        FR_CK(launch(s, c));
        ++cnt;
    }
    return enqueue_faces(s, s->parity, cnt);
}

// Adaptive steps: the first stage derivative k1 = R(u_n) of instances whose
// state was just set (accepted flag kAccFresh), before their first attempt;
// the others are left as they are.  Flips the face-buffer parity.
fr_status bs_start_if_needed(fr_solver *s) {
    if (!s->adapt || !s->bs_start) return FR_OK;
    int64_t cnt = 0;
    FR_TRY(enqueue_eval(s, s->parity, frk::M_BS_START, 0.0, 0.0, 0.0, cnt));
    s->parity ^= 1;
    s->bs_start = false;
    return FR_OK;
}

// One RK step starting from face-buffer parity p0; returns the launches issued.
fr_status enqueue_step(fr_solver *s, int p0, int64_t *n_launch) {
    if (s->adapt) return enqueue_attempt(s, p0, n_launch);
    int par = p0;
    int64_t cnt = 0;
    const int stages = s->cfg.rk == FR_RK4 ? 4 : 5;
    const double dt = s->cfg.dt;
    for (int st = 0; st < stages; ++st) {
        if (s->cfg.rk == FR_LSRK45) {
            FR_TRY(enqueue_eval(s, par, st == 0 ? frk::M_LSRK_FIRST : frk::M_LSRK, kLsA[st], kLsB[st], 0.0, cnt));
        } else {
            const int modes[4] = {frk::M_RK4_1, frk::M_RK4_2, frk::M_RK4_3, frk::M_RK4_4};
            const double cs[4] = {0.5 * dt, 0.5 * dt, dt, dt / 6.0};
            FR_TRY(enqueue_eval(s, par, modes[st], 0.0, 0.0, cs[st], cnt));
        }
        par ^= 1;
    }
    FR_TRY(enqueue_samples(s, par, cnt));
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
    if (s->visc && !s->fused) {
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
        f.kind = s->fused ? frk::K_STAGE : frk::K_FLUX;
        f.g = g;
        f.elem0 = s->grp[g].off[inst];
        f.n_elem = s->grp[g].ne[inst];
        f.UFin = s->grp[g].UF[s->parity];
        f.FVin = fvbuf(s->grp[g], s->parity);
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

// FP32 perturbation storage: the reference state and the FP64 constants
// derived from it.  u_ref is the configuration's free stream with each
// conserved component rounded to FP32, so that the stored perturbation plus
// u_ref is exactly the state the host sees.
void set_reference(fr_solver *s, const fr_config *cfg) {
    const int dim = s->dim, V = dim + 2;
    const double g = cfg->gamma;
    double m[3] = {0, 0, 0}, v2 = 0.0;
    for (int d = 0; d < dim; ++d) {
        m[d] = cfg->rho_inf * cfg->v_inf[d];
        v2 += cfg->v_inf[d] * cfg->v_inf[d];
    }
    s->uref64[0] = (double)(float)cfg->rho_inf;
    for (int d = 0; d < dim; ++d) s->uref64[1 + d] = (double)(float)m[d];
    s->uref64[V - 1] = (double)(float)(cfg->p_inf / (g - 1.0) + 0.5 * cfg->rho_inf * v2);
    const double rho = s->uref64[0], E = s->uref64[V - 1];
    double vr[3] = {0, 0, 0}, ke = 0.0;
    for (int d = 0; d < dim; ++d) {
        vr[d] = s->uref64[1 + d] / rho;
        ke += 0.5 * s->uref64[1 + d] * vr[d];
    }
    const double p = (g - 1.0) * (E - ke), H = E + p;
    s->pref64 = p;
    frk::RefState<float> &r = s->ref32;
    r = frk::RefState<float>{};
    r.rho = (float)rho;
    for (int d = 0; d < dim; ++d) {
        r.m[d] = (float)s->uref64[1 + d];
        r.v[d] = (float)vr[d];
        s->vref64[d] = vr[d];
    }
    r.E = (float)E;
    r.p = (float)p;
    r.H = (float)H;
    r.ke = (float)ke;
    r.drho_inf = (float)(cfg->rho_inf - rho);
    r.dp_inf = (float)(cfg->p_inf - p);
    r.c_inf = (float)std::sqrt(g * cfg->p_inf / cfg->rho_inf);
    // F_ref,j = [m_j, m_i v_j + p delta_ij, v_j H]
    for (int j = 0; j < dim; ++j) {
        s->Fref[j][0] = s->uref64[1 + j];
        for (int i = 0; i < dim; ++i) s->Fref[j][1 + i] = s->uref64[1 + i] * vr[j] + (i == j ? p : 0.0);
        s->Fref[j][V - 1] = vr[j] * H;
    }
}

// J times the FR residual of the constant reference flux F(u_ref) in degree
// group g (FP64): the divergence through the folded operator DT of the
// transformed reference flux S F_ref along every line plus g' times the
// reference part of the common fluxes, n F_ref at the element's own flux
// points and, on the lower side of a mortar face, minus the projection P of
// the higher side's n F_ref (what the kernels subtract there).  It vanishes
// to round-off wherever the discrete metric identities hold; the return
// value says whether it does not anywhere in the group.
bool reference_divergence(const fr_solver *s, int g, const std::vector<double> &met,
                          const std::vector<std::vector<double>> &nrm_groups, const std::vector<int32_t> &part,
                          const std::vector<frk::MortarFace> &mfaces, const std::vector<double> &mats,
                          std::vector<float> &out) {
    const std::vector<double> &nrm = nrm_groups[g];
    const Group &G = s->grp[g];
    const int dim = s->dim, V = s->V, MS = s->MS, N = G.N, nsp = G.nsp, nfp = G.nfp, nfpf = G.nfpf;
    const RefElem &r = G.ref;
    double DT[kMaxN][kMaxN];
    for (int i = 0; i < N; ++i)
        for (int mm = 0; mm < N; ++mm) DT[i][mm] = r.D1[i][mm] - r.dgR[i] * r.lend[1][mm] - r.dgL[i] * r.lend[0][mm];
    // lower-side mortar rows of this group: face and lane
    std::vector<std::pair<int64_t, int>> lo_row((size_t)G.n_box_lo, {-1, 0});
    for (size_t mi = 0; mi < mfaces.size(); ++mi) {
        const frk::MortarFace &F = mfaces[mi];
        if (F.glo != g) continue;
        for (int l = 0; l < F.nlo; ++l) lo_row[(size_t)(F.lo_box - G.fp_real + l)] = {(int64_t)mi, l};
    }
    auto stride = [&](int k) { return k == 0 ? 1 : (k == 1 ? N : N * N); };
    auto digit = [&](int sp, int k) { return (sp / stride(k)) % N; };
    auto fp_of = [&](int sp, int k, int side) {
        int l;
        if (dim == 2) {
            l = digit(sp, 1 - k);
        } else {
            const int a = (k == 0) ? 1 : 0, b = (k == 2) ? 1 : 2;
            l = digit(sp, a) + N * digit(sp, b);
        }
        return (2 * k + side) * nfpf + l;
    };
    out.assign((size_t)G.E * nsp * V, 0.0f);
    double worst = 0.0;
#pragma omp parallel for schedule(static) reduction(max : worst)
    for (int64_t e = 0; e < G.E; ++e) {
        // reference part of the common flux at every flux point of e
        std::vector<double> jref((size_t)nfp * V), fhat((size_t)nsp * dim * V);
        for (int f = 0; f < nfp; ++f) {
            const int32_t pt = part[(size_t)e * nfp + f];
            for (int v = 0; v < V; ++v) {
                double t = 0.0;
                if (pt >= G.fp_real && pt < G.fp_real + G.n_box_lo) {
                    const auto &fl = lo_row[(size_t)(pt - G.fp_real)];
                    const frk::MortarFace &F = mfaces[(size_t)fl.first];
                    const double *Pm = mats.data() + F.mat + (int64_t)F.nhi * F.nlo;
                    const std::vector<double> &nh = nrm_groups[F.ghi];
                    for (int l = 0; l < F.nhi; ++l) {
                        double nf = 0.0;
                        for (int j = 0; j < dim; ++j) nf += nh[(size_t)(F.hi_fp + l) * dim + j] * s->Fref[j][v];
                        t -= Pm[fl.second * F.nhi + l] * nf;
                    }
                } else {
                    for (int j = 0; j < dim; ++j) t += nrm[((size_t)e * nfp + f) * dim + j] * s->Fref[j][v];
                }
                jref[(size_t)f * V + v] = t;
            }
        }
        for (int sp = 0; sp < nsp; ++sp)
            for (int k = 0; k < dim; ++k)
                for (int v = 0; v < V; ++v) {
                    double t = 0.0;
                    for (int j = 0; j < dim; ++j)
                        t += met[((size_t)e * nsp + sp) * MS + k * dim + j] * s->Fref[j][v];
                    fhat[((size_t)sp * dim + k) * V + v] = t;
                }
        for (int sp = 0; sp < nsp; ++sp) {
            for (int v = 0; v < V; ++v) {
                double acc = 0.0, mag = 0.0;
                for (int k = 0; k < dim; ++k) {
                    const int ik = digit(sp, k), st = stride(k), q0 = sp - ik * st;
                    for (int mm = 0; mm < N; ++mm) {
                        const double t = DT[ik][mm] * fhat[((size_t)(q0 + mm * st) * dim + k) * V + v];
                        acc += t;
                        mag += std::fabs(t);
                    }
                    const double tp = r.dgR[ik] * jref[(size_t)fp_of(sp, k, 1) * V + v];
                    const double tm = -r.dgL[ik] * jref[(size_t)fp_of(sp, k, 0) * V + v];
                    acc += tp + tm;
                    mag += std::fabs(tp) + std::fabs(tm);
                }
                out[((size_t)e * nsp + sp) * V + v] = (float)acc;
                if (mag > 0.0) worst = std::max(worst, std::fabs(acc) / mag);
            }
        }
    }
    // round-off of the FP64 sums (a few dozen terms) stays far below this
    return worst > 1e-11;
}

}  // namespace
}  // namespace fr

using namespace fr;

extern "C" const char *fr_last_error(void) { return fr::g_last_error.c_str(); }

extern "C" size_t fr_workspace_bytes(fr_mesh *const *meshes, int n_inst, const fr_config *cfg) {
    if (check_batch(meshes, n_inst, cfg) != FR_OK) return 0;
    const Plan P = make_plan(meshes, n_inst);
    if (P.G > frk::kMaxGroups) return 0;
    return make_layout(P, n_inst, cfg->precision == FR_FP64, cfg->viscous != 0, cfg->rk == FR_BS32).total;
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
    s->adapt = cfg->rk == FR_BS32;
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
    const Layout L = make_layout(P, n_inst, s->fp64, s->visc, s->adapt);
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
        G.DIVREF = w + gl.DIVREF;
        G.FV2 = w + gl.FV2;
        G.LFP = w + gl.LFP;
        G.R3 = w + gl.R3;
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
    s->FLAGS = (int32_t *)(w + L.FLAGS);
    s->MATS = w + L.MATS;
    s->ERRE = (double *)(w + L.ERRE);
    s->ADAPT = (double *)(w + L.ADAPT);
    s->ACC = (int32_t *)(w + L.ACC);
    s->ARANGE = (frk::AdaptRange *)(w + L.ARANGE);

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

    if (!s->fp64) set_reference(s.get(), cfg);
    s->local_ref = cfg->flux_reference == 0;
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
    s->wall_nsum.assign((size_t)n_inst * 3, 0.0);
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
                    if (m->bctag[lf] == FR_TAG_WALL) {
                        // face quadrature weight: product of the free directions' weights
                        const int l = f % G.nfpf, n1 = G.N;
                        const double wf = dim == 2 ? G.ref.w[l] : G.ref.w[l % n1] * G.ref.w[l / n1];
                        for (int d = 0; d < dim; ++d) s->wall_nsum[(size_t)i * 3 + d] += wf * m->nrm[lf * dim + d];
                    }
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
                        // FP32 stores it relative to the reference velocity
                        for (int d = 0; d < dim; ++d)
                            bvref[(size_t)b * dim + d] = cfg->v_inf[d] * prof - s->vref64[d];
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
        if (s->visc) {
            FR_CK(cudaMemsetAsync(G.FV, 0, fc_bytes, cs));
            FR_CK(cudaMemsetAsync(G.FV2, 0, fc_bytes, cs));
        }
        FR_CK(cudaMemsetAsync(G.MFLUX, 0, (size_t)G.n_box * s->V * s->rsz, cs));
    }
    // BR2 stages may run as one fused kernel when every face is conforming;
    // the default is the gradient + flux kernel pair, fr_tune measures both
    const bool fusable = s->visc && cfg->viscous_scheme == FR_VISC_BR2 && P.n_mortar == 0;
    s->fused = false;
    if (fusable) {
        // partner lifting coefficients per own flux point (FP64, then cast):
        // lf = sum_m l_m(side) g'_side(m) (1/J) S[k][:] along the partner's line
        for (int g = 0; g < P.G; ++g) {
            const Group &G = s->grp[g];
            const RefElem &r = G.ref;
            const int nsp = G.nsp, nfp = G.nfp, N = G.N;
            std::vector<double> lf((size_t)G.E * nfp * dim, 0.0), lfp((size_t)G.E * nfp * dim, 0.0);
#pragma omp parallel for schedule(static)
            for (int64_t e = 0; e < G.E; ++e)
                for (int f = 0; f < nfp; ++f) {
                    const int k = r.fp_dir[f], side = r.fp_side[f];
                    for (int mm = 0; mm < N; ++mm) {
                        const int sp = ref_line_sp(r, f, mm);
                        const double *Mv = &met[g][((size_t)e * nsp + sp) * MS];
                        const double c = r.lend[side][mm] * (side ? r.dgR[mm] : r.dgL[mm]) * Mv[dim * dim];
                        for (int jd = 0; jd < dim; ++jd) lf[((size_t)e * nfp + f) * dim + jd] += c * Mv[k * dim + jd];
                    }
                }
            for (size_t q = 0; q < (size_t)G.E * nfp; ++q) {
                const int32_t pt = part[g][q];
                if (pt < 0) continue;
                for (int jd = 0; jd < dim; ++jd) lfp[q * dim + jd] = lf[(size_t)pt * dim + jd];
            }
            FR_CK(up_real(G.LFP, lfp, lfp.size()));
        }
    }
    if (!s->fp64) {
        std::vector<float> dr;
        for (int g = 0; g < P.G; ++g) {
            Group &G = s->grp[g];
            G.use_divref = reference_divergence(s.get(), g, met[g], nrm, part[g], mfaces, mats, dr);
            if (G.use_divref) FR_CK(up(G.DIVREF, dr.data(), dr.size() * sizeof(float)));
        }
    }
    FR_CK(up_real(s->BVREF, bvref, (size_t)P.nb * dim));
    FR_CK(up(s->BTAG, btag.data(), (size_t)P.nb * 4));
    FR_CK(up(s->MORT, mfaces.data(), mfaces.size() * sizeof(frk::MortarFace)));
    FR_CK(up_real(s->MATS, mats, (size_t)P.mat_reals));
    FR_CK(cudaMemsetAsync(s->pacc, 0, sizeof(frk::ProbeAcc) * kMaxProbes, cs));
    FR_CK(cudaMemsetAsync(s->force_acc, 0, (size_t)n_inst * 3 * 8, cs));
    FR_CK(cudaMemsetAsync(s->FLAGS, 0, (size_t)n_inst * 4, cs));
    if (s->adapt) {
        // per-element error sums: the groups one after another; every
        // instance's element ranges in them and its number of values
        int64_t base = 0;
        for (int g = 0; g < P.G; ++g) {
            s->grp[g].ebase = base;
            base += s->grp[g].E;
        }
        std::vector<frk::AdaptRange> ar(n_inst);
        for (int i = 0; i < n_inst; ++i) {
            std::memset(&ar[i], 0, sizeof(ar[i]));
            for (int g = 0; g < P.G; ++g) {
                ar[i].start[g] = s->grp[g].ebase + s->grp[g].off[i];
                ar[i].count[g] = s->grp[g].ne[i];
            }
            ar[i].nval = (double)s->inst_nsp[i] * s->V;
        }
        FR_CK(up(s->ARANGE, ar.data(), ar.size() * sizeof(frk::AdaptRange)));
        s->adapt_init.assign((size_t)n_inst * frk::kAdStride, 0.0);
        for (int i = 0; i < n_inst; ++i) {
            double *rec = &s->adapt_init[(size_t)i * frk::kAdStride];
            rec[frk::kAdH] = cfg->dt;
            rec[frk::kAdHuse] = first_step(*cfg);
        }
        FR_CK(up(s->ADAPT, s->adapt_init.data(), s->adapt_init.size() * 8));
        const std::vector<int32_t> fresh(n_inst, frk::kAccFresh);
        FR_CK(up(s->ACC, fresh.data(), fresh.size() * 4));
        s->bs_start = true;
    }
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
    if (s->xfer) {
        cudaStreamSynchronize(s->xfer);
        cudaStreamDestroy(s->xfer);
    }
    for (cudaEvent_t e : s->xev)
        if (e) cudaEventDestroy(e);
    delete s;
}

namespace {

// Adaptive steps: instance inst (-1: every instance) restarts at t = 0 with
// the first step of the configuration, its k1 still to be computed.
const int32_t kFreshFlag = frk::kAccFresh;
fr_status reset_step_control(fr_solver *s, int inst) {
    const int i0 = inst < 0 ? 0 : inst, i1 = inst < 0 ? s->n_inst : inst + 1;
    for (int i = i0; i < i1; ++i) {
        FR_CK(cudaMemcpyAsync(s->ADAPT + (size_t)i * frk::kAdStride, &s->adapt_init[(size_t)i * frk::kAdStride],
                              frk::kAdStride * 8, cudaMemcpyHostToDevice, s->stream));
        FR_CK(cudaMemcpyAsync(s->ACC + i, &kFreshFlag, 4, cudaMemcpyHostToDevice, s->stream));
    }
    s->bs_start = true;
    return FR_OK;
}

// Enqueue the upload of one instance's FP64 host state (the ABI's element
// order) and the derivation of its face values; no synchronisation.  An
// instance spread over several degree groups is reordered on the host into
// `tmp`, which must stay alive until the stream has been synchronised.
fr_status enqueue_upload(fr_solver *s, int inst, const double *u, std::vector<double> &tmp) {
    const int V = s->V;
    FR_CK(cudaMemsetAsync(s->FLAGS + inst, 0, 4, s->stream));
    if (s->adapt) FR_TRY(reset_step_control(s, inst));
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
        in.kind = s->fused ? frk::K_INTERP_VISC : frk::K_INTERP;
        in.g = (int)g;
        in.elem0 = G.off[inst];
        in.n_elem = G.ne[inst];
        in.UFout = G.UF[s->parity];
        in.FVout = fvbuf(G, s->parity);
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

// Whole-batch staging (every instance in one degree group, the usual case):
// one copy of all instances' FP64 states each way through the FP64 staging
// buffer, which holds the batch in the ABI's order; the conversions run over
// runs of instances that are consecutive both there and in their group.
bool batch_stageable(const fr_solver *s) {
    for (int i = 0; i < s->n_inst; ++i)
        if (spread(s, i)) return false;
    return true;
}

// Runs of consecutive instances in [i0, i1) that are consecutive both in the
// staging buffer and in their degree group: fn(group, first element, elements,
// staging offset in doubles).
template <typename F>
fr_status for_instance_runs(const fr_solver *s, int i0, int i1, F &&fn) {
    const int V = s->V;
    int g_run = -1;
    int64_t e0 = 0, ne = 0, so = 0, off = 0;
    for (int i = 0; i < i0; ++i) off += s->inst_nsp[i] * V;
    for (int i = i0; i <= i1; ++i) {
        int g = -1;
        if (i < i1)
            for (size_t h = 0; h < s->grp.size(); ++h)
                if (s->grp[h].ne[i] > 0) g = (int)h;
        const bool extend = i < i1 && g == g_run && s->grp[g].off[i] == e0 + ne &&
                            off == so + ne * s->grp[g].nsp * V;
        if (!extend) {
            if (g_run >= 0 && ne > 0) FR_TRY(fn(g_run, e0, ne, so));
            if (i < i1) {
                g_run = g;
                e0 = g >= 0 ? s->grp[g].off[i] : 0;
                ne = 0;
                so = off;
            }
        }
        if (i < i1) {
            if (g >= 0) ne += s->grp[g].ne[i];
            off += s->inst_nsp[i] * V;
        }
    }
    return FR_OK;
}

// Instance chunks of a batch transfer (up to kXferChunks, balanced by size):
// instance range [i0, i1), staging offset and length in doubles.
constexpr int kXferChunks = 4;
struct XferChunk { int i0, i1; int64_t off, n; };

std::vector<XferChunk> xfer_chunks(const fr_solver *s) {
    int64_t total = 0;
    for (int i = 0; i < s->n_inst; ++i) total += s->inst_nsp[i] * s->V;
    const int k = std::min(kXferChunks, s->n_inst);
    std::vector<XferChunk> out;
    int64_t off = 0;
    int i = 0;
    for (int c = 0; c < k && i < s->n_inst; ++c) {
        const int64_t goal = total * (c + 1) / k;
        XferChunk x{i, i, off, 0};
        while (i < s->n_inst && (off < goal || x.i1 == x.i0)) {
            const int64_t n = s->inst_nsp[i] * s->V;
            off += n;
            x.n += n;
            x.i1 = ++i;
        }
        out.push_back(x);
    }
    if (i < s->n_inst) {   // (rounding) the rest joins the last chunk
        for (; i < s->n_inst; ++i) out.back().n += s->inst_nsp[i] * s->V;
        out.back().i1 = s->n_inst;
    }
    return out;
}

cudaError_t ensure_xfer(fr_solver *s) {
    if (s->xfer) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&s->xfer, cudaStreamNonBlocking);
    for (int c = 0; c <= kXferChunks && e == cudaSuccess; ++c)
        e = cudaEventCreateWithFlags(&s->xev[c], cudaEventDisableTiming);
    return e;
}

// face data of the instances [i0, i1) (each in one degree group)
fr_status enqueue_faces_of(fr_solver *s, int i0, int i1) {
    for (size_t g = 0; g < s->grp.size(); ++g) {
        const Group &G = s->grp[g];
        int first = -1, last = -1;
        for (int i = i0; i < i1; ++i)
            if (G.ne[i] > 0) {
                if (first < 0) first = i;
                last = i;
            }
        if (first < 0) continue;
        Launch in;
        in.kind = s->fused ? frk::K_INTERP_VISC : frk::K_INTERP;
        in.g = (int)g;
        in.elem0 = G.off[first];
        in.n_elem = G.off[last] + G.ne[last] - G.off[first];
        in.UFout = G.UF[s->parity];
        in.FVout = fvbuf(G, s->parity);
        FR_CK(launch(s, in));
    }
    return FR_OK;
}

// Upload of the whole batch: chunk c's host-link copy runs on the auxiliary
// stream while the solver's stream converts chunk c - 1 and derives its face
// data.  The copies start after the solver stream's earlier work (which may
// still read the staging buffer).
fr_status enqueue_upload_batch(fr_solver *s, const double *u) {
    FR_CK(cudaMemsetAsync(s->FLAGS, 0, (size_t)s->n_inst * 4, s->stream));
    if (s->adapt) FR_TRY(reset_step_control(s, -1));
    FR_CK(ensure_xfer(s));
    const std::vector<XferChunk> ch = xfer_chunks(s);
    FR_CK(cudaEventRecord(s->xev[kXferChunks], s->stream));
    FR_CK(cudaStreamWaitEvent(s->xfer, s->xev[kXferChunks], 0));
    for (size_t c = 0; c < ch.size(); ++c) {
        FR_CK(cudaMemcpyAsync(s->stage64 + ch[c].off, u + ch[c].off, (size_t)ch[c].n * 8,
                              cudaMemcpyHostToDevice, s->xfer));
        FR_CK(cudaEventRecord(s->xev[c], s->xfer));
    }
    for (size_t c = 0; c < ch.size(); ++c) {
        FR_CK(cudaStreamWaitEvent(s->stream, s->xev[c], 0));
        FR_TRY(for_instance_runs(s, ch[c].i0, ch[c].i1, [&](int g, int64_t e0, int64_t ne, int64_t so) -> fr_status {
            Launch cv;
            cv.kind = frk::K_TO_REAL;
            cv.g = g;
            cv.elem0 = e0;
            cv.n_elem = ne;
            cv.stage_off = so;
            cv.grid = grid_for(ne * s->grp[g].nsp * s->V);
            FR_CK(launch(s, cv));
            return FR_OK;
        }));
        FR_TRY(enqueue_faces_of(s, ch[c].i0, ch[c].i1));
    }
    return FR_OK;
}

// Download of the whole batch: chunk c's conversion on the solver stream,
// its host-link copy on the auxiliary stream (overlapping the conversion of
// chunk c + 1); the solver stream then waits for the last copy.
fr_status enqueue_download_batch(fr_solver *s, int src, double *u) {
    FR_CK(ensure_xfer(s));
    const std::vector<XferChunk> ch = xfer_chunks(s);
    for (size_t c = 0; c < ch.size(); ++c) {
        FR_TRY(for_instance_runs(s, ch[c].i0, ch[c].i1, [&](int g, int64_t e0, int64_t ne, int64_t so) -> fr_status {
            Launch cv;
            cv.kind = frk::K_TO_F64;
            cv.g = g;
            cv.elem0 = e0;
            cv.n_elem = ne;
            cv.integral_src = src;
            cv.stage_off = so;
            cv.grid = grid_for(ne * s->grp[g].nsp * s->V);
            FR_CK(launch(s, cv));
            return FR_OK;
        }));
        FR_CK(cudaEventRecord(s->xev[c], s->stream));
        FR_CK(cudaStreamWaitEvent(s->xfer, s->xev[c], 0));
        FR_CK(cudaMemcpyAsync(u + ch[c].off, s->stage64 + ch[c].off, (size_t)ch[c].n * 8,
                              cudaMemcpyDeviceToHost, s->xfer));
    }
    FR_CK(cudaEventRecord(s->xev[kXferChunks], s->xfer));
    FR_CK(cudaStreamWaitEvent(s->stream, s->xev[kXferChunks], 0));
    return FR_OK;
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
    if (batch_stageable(s)) {
        fr_status st = enqueue_upload_batch(s, u);
        cudaError_t e = cudaStreamSynchronize(s->stream);   // the host array must outlive the copy
        // (on an error return the solver stream may not have waited for every
        // copy already issued on the transfer stream)
        if (s->xfer) cudaStreamSynchronize(s->xfer);
        if (st != FR_OK) return st;
        FR_CK(e);
        return FR_OK;
    }
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
    if (batch_stageable(s)) {
        fr_status st = enqueue_download_batch(s, 0, u);
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (s->xfer) cudaStreamSynchronize(s->xfer);   // as in fr_set_states
        if (st != FR_OK) return st;
        FR_CK(e);
        return FR_OK;
    }
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
    const int flips = step_flips(s);
    int64_t total = 0;
    if (n_steps > 0) FR_TRY(bs_start_if_needed(s));
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
        s->parity = (flips % 2) ? p0 ^ 1 : p0;
        ++s->steps_since_reset;
        if (s->cfg.check_every > 0 && ++s->steps_since_check >= s->cfg.check_every) {
            s->steps_since_check = 0;
            for (size_t g = 0; g < s->grp.size(); ++g) {
                Launch c;
                c.kind = frk::K_FINITE;
                c.g = (int)g;
                c.n_elem = s->grp[g].E;
                c.grid = grid_for(s->grp[g].E * s->grp[g].nsp);
                FR_CK(launch(s, c));
                ++total;
            }
        }
    }
    if (s->adapt && n_steps > 0) FR_TRY(bs_settle(s, total));
    s->last_launches = total;
    return FR_OK;
}

extern "C" fr_status fr_instance_status(fr_solver *s, int32_t *flags, int *first_bad) {
    fr::Range nvtx_range("fr_instance_status");
    if (!s || !first_bad) { set_error("null argument"); return FR_ERR_INVALID_ARG; }
    std::vector<int32_t> h(s->n_inst);
    FR_CK(cudaMemcpyAsync(h.data(), s->FLAGS, h.size() * 4, cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    *first_bad = -1;
    for (int i = 0; i < s->n_inst; ++i) {
        if (flags) flags[i] = h[i];
        if (h[i] && *first_bad < 0) *first_bad = i;
    }
    if (*first_bad >= 0) {
        set_error("non-finite values in the state of instance " + std::to_string(*first_bad));
        return FR_ERR_NONFINITE;
    }
    return FR_OK;
}

extern "C" fr_status fr_step_control(fr_solver *s, int inst, double *out8) {
    fr_status st = check_inst(s, inst);
    if (st != FR_OK) return st;
    if (!s->adapt || !out8) {
        set_error(out8 ? "fr_step_control: the solver does not use adaptive steps" : "null output");
        return FR_ERR_INVALID_ARG;
    }
    FR_CK(cudaMemcpyAsync(out8, s->ADAPT + (size_t)inst * frk::kAdStride, frk::kAdStride * 8,
                          cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    return FR_OK;
}

extern "C" fr_status fr_set_end_time(fr_solver *s, double t_end) {
    if (!s) { set_error("null solver"); return FR_ERR_INVALID_ARG; }
    if (!s->adapt || std::isnan(t_end)) {
        set_error(s->adapt ? "fr_set_end_time: invalid end time" : "fr_set_end_time: the solver does not use adaptive steps");
        return FR_ERR_INVALID_ARG;
    }
    s->cfg.t_end = t_end;
    // every instance's next step under the new end time (the rule of K_BS_CONTROL)
    const size_t n = (size_t)s->n_inst * frk::kAdStride;
    std::vector<double> rec(n);
    FR_CK(cudaMemcpyAsync(rec.data(), s->ADAPT, n * 8, cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    const double te = eff_t_end(s->cfg), hm = eff_dt_max(s->cfg);
    for (int i = 0; i < s->n_inst; ++i) {
        double *r = &rec[(size_t)i * frk::kAdStride];
        double h = std::min(r[frk::kAdH], hm);
        if (r[frk::kAdT] + h > te) h = te - r[frk::kAdT];
        r[frk::kAdHuse] = std::max(h, 0.0);
    }
    FR_CK(cudaMemcpyAsync(s->ADAPT, rec.data(), n * 8, cudaMemcpyHostToDevice, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    // the initial record of a state set later ends at the new time too
    for (int i = 0; i < s->n_inst; ++i) s->adapt_init[(size_t)i * frk::kAdStride + frk::kAdHuse] = first_step(s->cfg);
    drop_graphs(s);   // the captured attempts carry the end time
    return FR_OK;
}

extern "C" int64_t fr_last_launch_count(const fr_solver *s) { return s ? s->last_launches : -1; }

extern "C" fr_status fr_profile_steps(fr_solver *s, int n_steps, double *ms, int64_t *count) {
    fr::Range nvtx_range("fr_profile_steps");
    if (!s || n_steps <= 0 || !ms || !count) { set_error("invalid fr_profile_steps arguments"); return FR_ERR_INVALID_ARG; }
    const int flips = step_flips(s);
    FR_TRY(bs_start_if_needed(s));
    s->prof.clear();
    s->profiling = true;
    fr_status st = FR_OK;
    for (int it = 0; it < n_steps && st == FR_OK; ++it) {
        int64_t cnt = 0;
        st = enqueue_step(s, s->parity, &cnt);
        s->parity = (flips % 2) ? s->parity ^ 1 : s->parity;
        ++s->steps_since_reset;
    }
    s->profiling = false;
    int64_t settle_launches = 0;
    if (st == FR_OK && s->adapt) st = bs_settle(s, settle_launches);
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
    s->probe_elem.push_back(d.elem);
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

// Accumulator checkpoint: [steps in the window, number of probes, number of
// instances, probe fingerprint, wall-force sums n_inst x 3, probe
// accumulators n_probe x 16, sample rings n_probe x kHistLen]
static constexpr int kAccHeader = 4;

// identifies the observers (instance and element of each, in order); an
// integer below 2^53, so it survives the round trip through a double exactly
static double probe_fingerprint(const fr_solver *s) {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < s->n_probe; ++i) {
        h = (h ^ (uint64_t)s->probe_inst[i]) * 1099511628211ull;
        h = (h ^ (uint64_t)s->probe_elem[i]) * 1099511628211ull;
    }
    return (double)(h >> 11);
}

extern "C" int64_t fr_accumulators_size(const fr_solver *s) {
    if (!s) return -1;
    return kAccHeader + (int64_t)s->n_inst * 3 + (int64_t)s->n_probe * (int64_t)(sizeof(frk::ProbeAcc) / 8) +
           (int64_t)s->n_probe * frk::kHistLen + (s->adapt ? (int64_t)s->n_inst * frk::kAdStride : 0);
}

extern "C" fr_status fr_get_accumulators(fr_solver *s, double *out) {
    if (!s || !out) { set_error("null argument"); return FR_ERR_INVALID_ARG; }
    const size_t na = sizeof(frk::ProbeAcc) / 8;
    out[0] = (double)s->steps_since_reset;
    out[1] = (double)s->n_probe;
    out[2] = (double)s->n_inst;
    out[3] = probe_fingerprint(s);
    double *f = out + kAccHeader, *pa = f + (size_t)s->n_inst * 3, *ph = pa + (size_t)s->n_probe * na;
    FR_CK(cudaMemcpyAsync(f, s->force_acc, (size_t)s->n_inst * 3 * 8, cudaMemcpyDeviceToHost, s->stream));
    if (s->n_probe > 0) {
        FR_CK(cudaMemcpyAsync(pa, s->pacc, (size_t)s->n_probe * sizeof(frk::ProbeAcc), cudaMemcpyDeviceToHost,
                              s->stream));
        FR_CK(cudaMemcpyAsync(ph, s->phist, (size_t)s->n_probe * frk::kHistLen * 8, cudaMemcpyDeviceToHost,
                              s->stream));
    }
    if (s->adapt)
        FR_CK(cudaMemcpyAsync(ph + (size_t)s->n_probe * frk::kHistLen, s->ADAPT,
                              (size_t)s->n_inst * frk::kAdStride * 8, cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    return FR_OK;
}

extern "C" fr_status fr_set_accumulators(fr_solver *s, const double *in, int64_t n) {
    if (!s || !in) { set_error("null argument"); return FR_ERR_INVALID_ARG; }
    if (n != fr_accumulators_size(s)) {
        set_error("accumulator checkpoint has " + std::to_string(n) + " values, this solver's has " +
                  std::to_string(fr_accumulators_size(s)));
        return FR_ERR_INVALID_ARG;
    }
    if (in[1] != (double)s->n_probe || in[2] != (double)s->n_inst || !(in[0] >= 0.0)) {
        set_error("accumulator checkpoint is for " + std::to_string((int64_t)in[2]) + " instances and " +
                  std::to_string((int64_t)in[1]) + " probes, the solver has " + std::to_string(s->n_inst) +
                  " and " + std::to_string(s->n_probe));
        return FR_ERR_INVALID_ARG;
    }
    if (in[3] != probe_fingerprint(s)) {
        set_error("accumulator checkpoint was taken with other observers (instances or locations differ)");
        return FR_ERR_INVALID_ARG;
    }
    const size_t na = sizeof(frk::ProbeAcc) / 8;
    const double *f = in + kAccHeader, *pa = f + (size_t)s->n_inst * 3, *ph = pa + (size_t)s->n_probe * na;
    FR_CK(cudaMemcpyAsync(s->force_acc, f, (size_t)s->n_inst * 3 * 8, cudaMemcpyHostToDevice, s->stream));
    if (s->n_probe > 0) {
        FR_CK(cudaMemcpyAsync(s->pacc, pa, (size_t)s->n_probe * sizeof(frk::ProbeAcc), cudaMemcpyHostToDevice,
                              s->stream));
        FR_CK(cudaMemcpyAsync(s->phist, ph, (size_t)s->n_probe * frk::kHistLen * 8, cudaMemcpyHostToDevice,
                              s->stream));
    }
    if (s->adapt)
        FR_CK(cudaMemcpyAsync(s->ADAPT, ph + (size_t)s->n_probe * frk::kHistLen,
                              (size_t)s->n_inst * frk::kAdStride * 8, cudaMemcpyHostToDevice, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    s->steps_since_reset = (int64_t)in[0];
    return FR_OK;
}

extern "C" fr_status fr_probe_reset(fr_solver *s) {
    if (!s) { set_error("null solver"); return FR_ERR_INVALID_ARG; }
    FR_CK(cudaMemsetAsync(s->pacc, 0, sizeof(frk::ProbeAcc) * kMaxProbes, s->stream));
    FR_CK(cudaMemsetAsync(s->force_acc, 0, (size_t)s->n_inst * 3 * 8, s->stream));
    if (s->adapt)   // the accepted-step counters of the averaging window
        FR_CK(cudaMemset2DAsync(s->ADAPT + frk::kAdSamples, frk::kAdStride * 8, 0, 8, s->n_inst, s->stream));
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
    double h[3], samples = (double)s->steps_since_reset;
    FR_CK(cudaMemcpyAsync(h, s->force_acc + (size_t)inst * 3, 24, cudaMemcpyDeviceToHost, s->stream));
    if (s->adapt)   // adaptive steps: the instance's accepted steps in the window
        FR_CK(cudaMemcpyAsync(&samples, s->ADAPT + (size_t)inst * frk::kAdStride + frk::kAdSamples, 8,
                              cudaMemcpyDeviceToHost, s->stream));
    FR_CK(cudaStreamSynchronize(s->stream));
    const double n = std::max(samples, 1.0);
    for (int d = 0; d < s->dim; ++d) {
        mean_force[d] = h[d] / n;
        if (!s->fp64 && samples > 0) mean_force[d] += s->pref64 * s->wall_nsum[(size_t)inst * 3 + d];
    }
    return FR_OK;
}

extern "C" fr_status fr_force_coefficients(fr_solver *s, int inst, double a_ref, double *mean_cl,
                                           double *mean_cd) {
    if (!mean_cl || !mean_cd || !(a_ref > 0.0)) {
        set_error("invalid fr_force_coefficients arguments");
        return FR_ERR_INVALID_ARG;
    }
    double F[3] = {0, 0, 0};
    fr_status st = fr_forces(s, inst, F);
    if (st != FR_OK) return st;
    const int dim = s->dim;
    double vv = 0.0;
    for (int d = 0; d < dim; ++d) vv += s->cfg.v_inf[d] * s->cfg.v_inf[d];
    if (!(vv > 0.0) || !(s->cfg.rho_inf > 0.0)) {
        set_error("force coefficients need a non-zero free-stream velocity");
        return FR_ERR_INVALID_ARG;
    }
    const double vm = std::sqrt(vv);
    double dr[3] = {0, 0, 0}, li[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) dr[d] = s->cfg.v_inf[d] / vm;
    if (dim == 2) {
        li[0] = -dr[1];
        li[1] = dr[0];
    } else {
        // the y axis made orthogonal to the drag direction
        for (int d = 0; d < 3; ++d) li[d] = (d == 1 ? 1.0 : 0.0) - dr[1] * dr[d];
        const double ln = std::sqrt(li[0] * li[0] + li[1] * li[1] + li[2] * li[2]);
        if (!(ln > 1e-12)) { set_error("free stream along the y axis: lift direction undefined"); return FR_ERR_INVALID_ARG; }
        for (int d = 0; d < 3; ++d) li[d] /= ln;
    }
    const double q = 0.5 * s->cfg.rho_inf * vv * a_ref;
    double cl = 0.0, cd = 0.0;
    for (int d = 0; d < dim; ++d) {
        cl += F[d] * li[d];
        cd += F[d] * dr[d];
    }
    *mean_cl = cl / q;
    *mean_cd = cd / q;
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

// Device address of the scratch array on the current device, looked up on
// every call (cudaGetSymbolAddress, with the caller's device current): a
// cached address would outlive a device reset or a re-created primary
// context, and the lookup costs far less than the launches it serves.
fr_status static_scratch(double **out) {
    void *p = nullptr;
    FR_CK(cudaGetSymbolAddress(&p, g_static_scratch));
    *out = static_cast<double *>(p);
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

// --------------------------------------------------------------------------
// Autotuner (fr_tune): the stage schedule of a solver (BR2: one fused kernel
// or gradient + flux kernels) and the register level of its stage kernels,
// measured on the solver's own batch and cached in a small JSON file keyed
// on the GPU architecture and the batch's shape.
// --------------------------------------------------------------------------
namespace fr {
namespace {

std::string schedule_string(const fr_solver *s) {
    char buf[192];
    std::snprintf(buf, sizeof(buf), "stage=%s;regs=%d;contract=%s;ms=%.6f;source=%s", s->fused ? "fused" : "split",
                  s->regs_level, s->tc ? "tc" : "simt", s->schedule_ms, s->schedule_source.c_str());
    return buf;
}

std::string tune_key(const fr_solver *s) {
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) == cudaSuccess) cudaGetDeviceProperties(&prop, dev);
    int64_t nsp = 0;
    std::string deg;
    for (const Group &G : s->grp) {
        nsp += G.E * G.nsp;
        if (!deg.empty()) deg += ",";
        deg += std::to_string(G.p);
    }
    int bucket = 0;
    while (((int64_t)1 << (bucket + 1)) <= nsp) ++bucket;
    char buf[256];
    std::snprintf(buf, sizeof(buf), "sm_%d%d|dim=%d|p=%s|V=%d|%s|%s|%s|mortar=%d|log2sp=%d", prop.major,
                  prop.minor, s->dim, deg.c_str(), s->V, s->fp64 ? "fp64" : "fp32",
                  !s->visc ? "euler" : (s->cfg.viscous_scheme == FR_VISC_LDG ? "ldg" : "br2"),
                  s->cfg.flux == FR_FLUX_ROE ? "roe" : "rusanov", s->n_mortar > 0 ? 1 : 0, bucket);
    return buf;
}

// The cache file: a JSON object with one "key": "value" pair per line.
std::map<std::string, std::string> read_cache(const char *path) {
    std::map<std::string, std::string> m;
    if (!path) return m;
    FILE *f = std::fopen(path, "r");
    if (!f) return m;
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        std::string l(line);
        const size_t a = l.find('"');
        if (a == std::string::npos) continue;
        const size_t b = l.find('"', a + 1);
        if (b == std::string::npos) continue;
        const size_t c = l.find('"', b + 1);
        if (c == std::string::npos) continue;
        const size_t d = l.find('"', c + 1);
        if (d == std::string::npos) continue;
        if (l.find(':', b) > c) continue;
        m[l.substr(a + 1, b - a - 1)] = l.substr(c + 1, d - c - 1);
    }
    std::fclose(f);
    return m;
}

bool write_cache(const char *path, const std::map<std::string, std::string> &m) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : m) std::fprintf(f, "  \"%s\": \"%s\"%s\n", kv.first.c_str(), kv.second.c_str(), ++i < m.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

// apply "stage=...;regs=..." if it is valid for this solver
bool apply_schedule(fr_solver *s, const std::string &v, const char *source) {
    const bool fused = v.find("stage=fused") != std::string::npos;
    const size_t r = v.find("regs=");
    const int regs = r == std::string::npos ? 0 : std::atoi(v.c_str() + r + 5);
    const bool tc = v.find("contract=tc") != std::string::npos;
    const bool fusable = s->visc && s->cfg.viscous_scheme == FR_VISC_BR2 && s->n_mortar == 0;
    if ((fused && !fusable) || regs < 0 || regs >= frk::kRegLevels || (tc && s->fp64)) return false;
    s->fused = fused;
    // FP64 and adaptive steps run the stage kernels at register level 0 only
    s->regs_level = (s->fp64 || s->adapt) ? 0 : regs;
    s->tc = tc;
    const size_t m = v.find("ms=");
    s->schedule_ms = m == std::string::npos ? 0.0 : std::atof(v.c_str() + m + 3);
    s->schedule_source = source;
    drop_graphs(s);
    return true;
}

}  // namespace
}  // namespace fr

extern "C" fr_status fr_tune_lookup(const char *cache_path, const char *key, char *value, size_t len) {
    if (!cache_path || !key || !value || len == 0) { set_error("invalid fr_tune_lookup arguments"); return FR_ERR_INVALID_ARG; }
    const auto m = fr::read_cache(cache_path);
    const auto it = m.find(key);
    value[0] = 0;
    if (it == m.end()) { set_error("no cached schedule for this key"); return FR_ERR_INVALID_ARG; }
    std::snprintf(value, len, "%s", it->second.c_str());
    return FR_OK;
}

extern "C" fr_status fr_schedule(fr_solver *s, char *out, size_t len, char *key, size_t key_len) {
    if (!s) { set_error("null solver"); return FR_ERR_INVALID_ARG; }
    if (out && len) std::snprintf(out, len, "%s", fr::schedule_string(s).c_str());
    if (key && key_len) std::snprintf(key, key_len, "%s", fr::tune_key(s).c_str());
    return FR_OK;
}

extern "C" fr_status fr_tune(fr_solver *s, const char *cache_path, int mode, char *choice, size_t choice_len) {
    fr::Range nvtx_range("fr_tune");
    if (!s || mode < 0 || mode > 2) { set_error("invalid fr_tune arguments"); return FR_ERR_INVALID_ARG; }
    const std::string key = fr::tune_key(s);
    auto cache = fr::read_cache(cache_path);
    const auto hit = cache.find(key);
    if (mode != 1 && hit != cache.end() && fr::apply_schedule(s, hit->second, "cache")) {
        if (choice && choice_len) std::snprintf(choice, choice_len, "%s", fr::schedule_string(s).c_str());
        return FR_OK;
    }
    if (mode == 2) {   // lookup only: keep the default
        if (choice && choice_len) std::snprintf(choice, choice_len, "%s", fr::schedule_string(s).c_str());
        return FR_OK;
    }
    // candidates: stage schedule x register level
    struct Cand { bool fused; int regs; bool tc; double ms; };
    std::vector<Cand> cands;
    const bool fusable = s->visc && s->cfg.viscous_scheme == FR_VISC_BR2 && s->n_mortar == 0;
    for (int c = 0; c < (s->fp64 ? 1 : 2); ++c)
        for (int f = 0; f < (fusable ? 2 : 1); ++f)
            for (int r = 0; r < ((s->fp64 || s->adapt) ? 1 : frk::kRegLevels); ++r) cands.push_back({f == 1, r, c == 1, 0.0});
    const int warm = 2, timed = 3;
    const int flips = step_flips(s);
    // every instance starts from the free stream of the configuration
    {
        const int V = s->V;
        double u0[5] = {s->cfg.rho_inf, 0, 0, 0, 0}, v2 = 0.0;
        for (int d = 0; d < s->dim; ++d) {
            u0[1 + d] = s->cfg.rho_inf * s->cfg.v_inf[d];
            v2 += s->cfg.v_inf[d] * s->cfg.v_inf[d];
        }
        u0[V - 1] = s->cfg.p_inf / (s->cfg.gamma - 1.0) + 0.5 * s->cfg.rho_inf * v2;
        for (int i = 0; i < s->n_inst; ++i) {
            std::vector<double> fs((size_t)s->inst_nsp[i] * V), tmp;
            for (size_t q = 0; q < fs.size(); ++q) fs[q] = u0[q % V];
            fr_status su = enqueue_upload(s, i, fs.data(), tmp);
            if (su != FR_OK) return su;
            FR_CK(cudaStreamSynchronize(s->stream));
        }
    }
    cudaEvent_t e0, e1;
    FR_CK(cudaEventCreate(&e0));
    FR_CK(cudaEventCreate(&e1));
    fr_status st = FR_OK;
    for (Cand &c : cands) {
        s->fused = c.fused;
        s->regs_level = c.regs;
        s->tc = c.tc;
        drop_graphs(s);
        // face data for this schedule, then warm-up and timed steps
        for (int i = 0; i < s->n_inst && st == FR_OK; ++i) {
            for (size_t g = 0; g < s->grp.size(); ++g) {
                const Group &G = s->grp[g];
                if (G.ne[i] <= 0) continue;
                Launch in;
                in.kind = s->fused ? frk::K_INTERP_VISC : frk::K_INTERP;
                in.g = (int)g;
                in.elem0 = G.off[i];
                in.n_elem = G.ne[i];
                in.UFout = G.UF[s->parity];
                in.FVout = fvbuf(G, s->parity);
                if (launch(s, in) != cudaSuccess) st = FR_ERR_CUDA;
            }
            if (st == FR_OK && mortar(s, 0, s->parity, s->moff[i], s->mcnt[i]) != cudaSuccess) st = FR_ERR_CUDA;
        }
        if (st == FR_OK) st = bs_start_if_needed(s);
        for (int it = 0; it < warm + timed && st == FR_OK; ++it) {
            if (it == warm && cudaEventRecord(e0, s->stream) != cudaSuccess) st = FR_ERR_CUDA;
            int64_t cnt = 0;
            if (st == FR_OK) st = enqueue_step(s, s->parity, &cnt);
            s->parity = (flips % 2) ? s->parity ^ 1 : s->parity;
        }
        if (st == FR_OK && cudaEventRecord(e1, s->stream) != cudaSuccess) st = FR_ERR_CUDA;
        if (st == FR_OK && cudaEventSynchronize(e1) != cudaSuccess) st = FR_ERR_CUDA;
        float ms = 0.f;
        if (st == FR_OK) cudaEventElapsedTime(&ms, e0, e1);
        c.ms = ms / timed;
        if (st != FR_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the steps above ran on whatever state the solver held: start afresh
    cudaMemsetAsync(s->pacc, 0, sizeof(frk::ProbeAcc) * kMaxProbes, s->stream);
    cudaMemsetAsync(s->force_acc, 0, (size_t)s->n_inst * 3 * 8, s->stream);
    cudaMemsetAsync(s->FLAGS, 0, (size_t)s->n_inst * 4, s->stream);
    s->steps_since_reset = 0;
    if (st == FR_OK && s->adapt) st = reset_step_control(s, -1);
    if (st != FR_OK) {
        set_error("fr_tune: a candidate schedule failed to run");
        return st;
    }
    const Cand *best = &cands[0];
    for (const Cand &c : cands)
        if (c.ms < best->ms) best = &c;
    char v[160];
    std::snprintf(v, sizeof(v), "stage=%s;regs=%d;contract=%s;ms=%.6f", best->fused ? "fused" : "split", best->regs,
                  best->tc ? "tc" : "simt", best->ms);
    fr::apply_schedule(s, v, "measured");
    std::string all;
    for (const Cand &c : cands) {
        char b[96];
        std::snprintf(b, sizeof(b), "%s%s/%d/%s=%.4f", all.empty() ? "" : ",", c.fused ? "fused" : "split", c.regs,
                      c.tc ? "tc" : "simt", c.ms);
        all += b;
    }
    if (cache_path) {
        cache[key] = v;
        fr::write_cache(cache_path, cache);
    }
    if (choice && choice_len)
        std::snprintf(choice, choice_len, "%s;candidates=%s", fr::schedule_string(s).c_str(), all.c_str());
    return FR_OK;
}
