/*
 * fr.h - C ABI of the GB300 (sm_103a) Flux Reconstruction hot path.
 *
 * One design evaluation of the aeroacoustic shape-optimisation loop of
 * Hamedi & Vermeire, "Gradient-Free Aeroacoustic Shape Optimization Using
 * Large Eddy Simulation" (arXiv:2312.14167): the explicit high-order FR
 * residual of the compressible Navier-Stokes equations (Sec. 2.1, Eqs. 1-7;
 * FR discretisation Sec. 2.3) on unstructured quad / hex meshes, explicit
 * Runge-Kutta time stepping, the observer pressure probe and the OASPL
 * reduction (Sec. 3.1.2, Eqs. 9-12), with the candidate designs of one MADS
 * poll (Sec. 2.2, Algorithm 1: all candidates of an iteration evaluated
 * concurrently) advanced together as a batch on one GPU.
 *
 * Conventions shared by every entry point:
 *  - every call returns an fr_status; nothing aborts or throws across the
 *    ABI; fr_last_error() returns a message for the calling thread's last
 *    failure;
 *  - host arrays belong to the caller and are only read (inputs) or
 *    written (outputs) during the call;
 *  - device memory comes only from the caller's workspace (fr_solver_create);
 *    the library itself never allocates device memory;
 *  - work is issued on the caller's CUDA stream; calls that return host data
 *    synchronise that stream before returning;
 *  - state layout on the host is [element][solution point][variable] in
 *    FP64, variables [rho, rho*v_x, rho*v_y(, rho*v_z), rho*E]; on a mesh
 *    whose degree varies (fr_mesh_create_varp) each element contributes its
 *    own (p_e+1)^dim points, element after element;
 *  - solution points are the tensor product of the p+1 Gauss-Legendre
 *    points, xi index fastest; element corners in tensor order (xi fastest);
 *    faces numbered -xi, +xi, -eta, +eta(, -zeta, +zeta).
 */
#ifndef FR_H
#define FR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fr_status;
#define FR_OK 0
#define FR_ERR_INVALID_ARG 1   /* null pointer, out-of-range index or size */
#define FR_ERR_MESH 2          /* unmatched face, non-positive Jacobian, ... */
#define FR_ERR_UNSUPPORTED 3   /* p outside 0..4, mixed dimensions in a batch */
#define FR_ERR_CUDA 4          /* a CUDA runtime call failed */
#define FR_ERR_NONFINITE 5     /* NaN/Inf found in the state */
#define FR_ERR_TIMEOUT 6       /* reserved for a bounded device wait that gave up;
                                  no call returns it today (no kernel of this
                                  library waits on another) */
#define FR_ERR_WORKSPACE 7     /* workspace too small or misaligned */

/* face tags (fr_mesh_create) */
#define FR_TAG_INTERIOR 0   /* matched to the face with the same corner vertices */
#define FR_TAG_PERIODIC 1   /* matched after a +/- periodic shift */
#define FR_TAG_WALL 2       /* no-slip adiabatic wall (Sec. 3.1.1) */
#define FR_TAG_FARFIELD 3   /* characteristic (Riemann-invariant) far field */
#define FR_TAG_INFLOW 4     /* far field with a tanh boundary-layer profile */
#define FR_TAG_OUTFLOW 5    /* characteristic outflow (same construction) */

#define FR_RK4 0            /* classical 4-stage RK */
#define FR_LSRK45 1         /* Carpenter-Kennedy 5-stage 4th-order 2N-storage */
/* Adaptive steps.  The paper advances in time with a second-order scheme with
 * adaptive steps (Sec. 2.3) whose coefficients it does not give; in its place
 * this is the embedded 3(2) pair of Bogacki and Shampine (1989): third-order
 * solution, second-order error estimate, the last stage derivative reused as
 * the next step's first (three residual evaluations per attempt).  Every
 * instance has its own time and step size.  Error norm of an attempt: the
 * root mean square, over all of the instance's solution-point values, of
 * e / (atol_v + rtol max(|u_n|, |u_n+1|)) (full conserved values, v the
 * variable); accepted when below 1.  Next step: the elementary error-per-step
 * controller (Hairer, Norsett and Wanner, Solving ODEs I, Sec. II.4),
 * h_new = h min(10, max(0.2, 0.9 err^(-1/3))), the increase capped at 1 right
 * after a rejection within the same step; every step is capped at dt_max
 * and shortened to end exactly at t_end, after which the instance does
 * nothing.  The decisions are taken on the device in FP64.  cfg.dt is the
 * first proposed step; fr_rk_step(n) makes n attempts (accepted or not);
 * observers and wall forces sample after accepted steps only. */
#define FR_BS32 2

#define FR_FLUX_RUSANOV 0   /* local Lax-Friedrichs: max |v.n| + c of both sides */
#define FR_FLUX_ROE 1       /* Roe averages, Harten entropy fix on the acoustic waves */

/* viscous interface scheme.  BR2: face gradient = interpolated uncorrected
 * gradient + eta x lifting of that face's jump, central viscous flux.  LDG:
 * each interface has a fixed left side (the point with the smaller global
 * index, s = +1 there, -1 on the other side); common solution
 * (1/2 + s beta) u_own + (1/2 - s beta) u_other, face gradient = the corrected
 * gradient interpolated to the face, common viscous normal flux
 * (1/2 - s beta) F_own.n + (1/2 + s beta) F_other.n - tau |n| (u_own - u_other). */
#define FR_VISC_BR2 0
#define FR_VISC_LDG 1

#define FR_FP64 0           /* plain FP64 state, geometry and arithmetic */
#define FR_FP32 1           /* FP32 state/fluxes/contractions; geometry computed in
                               FP64 then cast; FP64 probe/force/conservation sums.
                               The device state is the FP32 perturbation
                               u - u_ref about the reference state u_ref =
                               (rho_inf, rho_inf v_inf, p_inf/(gamma-1) +
                               rho_inf |v_inf|^2 / 2), each component rounded
                               to FP32, and fluxes are evaluated as
                               F(u) - F(u_ref); the host sees full FP64 states
                               (u_ref + the stored perturbation) */

typedef struct fr_mesh fr_mesh;
typedef struct fr_solver fr_solver;

/* Physics, scheme and precision of one solver (all instances share it).
 * Non-dimensional: the caller chooses the reference scales. */
typedef struct fr_config {
    double gamma;          /* ratio of specific heats (Sec. 2.1: 1.4) */
    double prandtl;        /* Prandtl number (Sec. 2.1: 0.71) */
    double mu;             /* constant dynamic viscosity */
    double rho_inf;        /* reference (far-field) density */
    double v_inf[3];       /* reference velocity */
    double p_inf;          /* reference pressure */
    double inflow_delta;   /* FR_TAG_INFLOW: v = v_inf tanh(3 (y - ywall)/delta); <= 0: uniform */
    double inflow_ywall;
    double br2_eta;        /* BR2 penalty; <= 0 selects the number of element faces */
    double dt;             /* fixed time step of fr_rk_step (FR_BS32: the first proposed step) */
    int viscous;           /* 0: Euler, 1: Navier-Stokes (BR2) */
    int rk;                /* FR_RK4, FR_LSRK45 or FR_BS32 */
    int precision;         /* FR_FP64 or FR_FP32 */
    int flux;              /* inviscid interface flux: FR_FLUX_RUSANOV or FR_FLUX_ROE */
    int viscous_scheme;    /* FR_VISC_BR2 or FR_VISC_LDG */
    int check_every;       /* > 0: fr_rk_step scans every instance's state for
                              NaN/Inf after every check_every-th step and flags
                              the instances concerned (fr_instance_status); 0: off */
    double ldg_beta;       /* LDG: one-sidedness of the common solution (0.5: upwind) */
    double ldg_tau;        /* LDG: penalty on the solution jump */
    int flux_reference;    /* FP32: 0 = every element evaluates its fluxes as perturbations
                              about its own reference state (the state at its first solution
                              point; accurate near walls, where the flow is far from the free
                              stream); 1 = about the free stream everywhere (fewer
                              instructions, larger rounding in wall cells) */
    int reserved;
    /* FR_BS32 only */
    double t_end;          /* end time of every instance (<= 0: none) */
    double dt_max;         /* largest step (<= 0: none) */
    double rtol;           /* relative tolerance of the error norm (>= 0) */
    double atol[5];        /* absolute tolerance per conserved variable (rho, rho v, rho E;
                              >= 0, with atol_v + rtol > 0 for each variable used) */
} fr_config;

/* Build one mesh (host, FP64).  The FR discretisation is Huynh's Flux
 * Reconstruction (Sec. 2.3) with the DG-recovery correction; the mesh
 * determines solution/flux points, metric terms (adjugate of the Jacobian of
 * the element map), outward normals scaled by the surface Jacobian and the
 * partner of every flux point.
 *  dim            2 (quads) or 3 (hexes)
 *  p              polynomial degree, 0..4 (0: one solution point per element,
 *                 the first-order finite-volume limit of the scheme)
 *  xyz            n_vert * dim vertex coordinates
 *  elem_vert      n_elem * 2^dim corner vertex indices, tensor order
 *  geo_order      degree q >= 1 of the element map
 *  geo_nodes      NULL (straight-sided: corners) or n_elem * (q+1)^dim * dim
 *                 coordinates of the equispaced tensor lattice (xi fastest)
 *  face_tag       n_elem * 2*dim tags (FR_TAG_*)
 *  n_shift, periodic_shift  n_shift * dim translation vectors for periodic
 *                 faces (a periodic face matches the face whose corners equal
 *                 its own plus or minus one shift)
 * Errors: FR_ERR_INVALID_ARG, FR_ERR_UNSUPPORTED (p), FR_ERR_MESH (a face
 * without partner, flux points that do not coincide, J <= 0). */
fr_status fr_mesh_create(fr_mesh **out, int dim, int p, int64_t n_vert, const double *xyz,
                         int64_t n_elem, const int64_t *elem_vert, int geo_order,
                         const double *geo_nodes, const int32_t *face_tag, int n_shift,
                         const double *periodic_shift);
void fr_mesh_destroy(fr_mesh *mesh);
/* A mesh whose polynomial degree is chosen per element (Sec. 5.1: the
 * airfoil grids run with a variable solution degree, P0-P3 / P0-P4, lower
 * degrees in the outer zones to damp waves before the boundaries).  Same
 * arguments as fr_mesh_create with ``elem_p`` (n_elem degrees, 0..4) in place
 * of p.  The paper does not say how a face joining two degrees is treated;
 * this library uses the conservative mortar coupling: the mortar is the
 * higher side's set of flux points, the lower side's face trace is evaluated
 * there, the higher side's trace reaches the lower side as its L2 projection
 * onto the lower degree, the common normal flux is formed on the mortar and
 * the lower side receives minus its projection (which keeps the face
 * integral); on such a face the lower-degree side is LDG's left side.
 * Errors: as fr_mesh_create; FR_ERR_MESH also when the corners of a face
 * joining two degrees do not coincide. */
fr_status fr_mesh_create_varp(fr_mesh **out, int dim, const int32_t *elem_p, int64_t n_vert,
                              const double *xyz, int64_t n_elem, const int64_t *elem_vert,
                              int geo_order, const double *geo_nodes, const int32_t *face_tag,
                              int n_shift, const double *periodic_shift);
/* Number of elements, solution points per element and flux points per
 * element (nsp = nfp = 0 when the degree varies between elements). */
fr_status fr_mesh_info(const fr_mesh *mesh, int64_t *n_elem, int *nsp, int *nfp);
/* Degree of every element (elem_p: n_elem int32, may be NULL) and the total
 * number of solution points of the mesh (may be NULL). */
fr_status fr_mesh_degrees(const fr_mesh *mesh, int32_t *elem_p, int64_t *n_sol_points);
/* Physical coordinates of all solution points, element after element, FP64
 * (n_sol_points * dim values). */
fr_status fr_mesh_sol_coords(const fr_mesh *mesh, double *xyz);

/* Workspace (device bytes) a solver over these meshes needs; 0 on error. */
size_t fr_workspace_bytes(fr_mesh *const *meshes, int n_inst, const fr_config *cfg);

/* Create a batch solver: the n_inst meshes (same dim; degrees may differ
 * between and within meshes) are advanced together: the elements of each
 * degree form one group, one element tile table over all instances, and the
 * faces joining two degrees are coupled by mortar kernels.  ``workspace`` is a
 * device buffer of ``ws_bytes`` >= fr_workspace_bytes() aligned to 256 bytes,
 * owned by the caller and kept alive until fr_solver_destroy; ``stream`` is a
 * cudaStream_t (NULL: legacy default stream).  Meshes may be destroyed after
 * this call.  The state starts at zero; call fr_set_state for every instance. */
fr_status fr_solver_create(fr_solver **out, fr_mesh *const *meshes, int n_inst,
                           const fr_config *cfg, void *workspace, size_t ws_bytes,
                           void *stream);
void fr_solver_destroy(fr_solver *solver);

/* Copy one instance's state (host FP64 [elem][sp][var]) in / out.  Both
 * synchronise the solver's stream. */
fr_status fr_set_state(fr_solver *solver, int inst, const double *u);
fr_status fr_get_state(fr_solver *solver, int inst, double *u);
/* The states of all instances at once: u holds instance 0's state, then
 * instance 1's, ... (each in the layout of fr_set_state), sum over instances
 * of n_sol_points * V doubles.  When every instance lies in one degree group
 * (the usual case) the whole batch moves in one copy each way through the
 * workspace's FP64 staging area, converted by one launch per run of
 * consecutive instances; an instance with elements of several degrees goes
 * through a host reorder, one instance after another.  The stream is
 * synchronised once, which is what a poll evaluator that moves every
 * candidate each step wants; with pinned host memory the copies run at the
 * host link's speed.  Same results as one fr_set_state / fr_get_state per
 * instance.  Errors: FR_ERR_INVALID_ARG
 * (null pointer), FR_ERR_CUDA. */
fr_status fr_set_states(fr_solver *solver, const double *u);
fr_status fr_get_states(fr_solver *solver, double *u);

/* du/dt of the current state of instance ``inst`` at its solution points
 * (host FP64 [elem][sp][var]): the FR residual of Sec. 2.3 applied to
 * Eq. 1. */
fr_status fr_residual(fr_solver *solver, int inst, double *r);

/* Advance every instance by n_steps fixed steps of cfg->dt with cfg->rk,
 * sampling every probe (and the wall force) after each completed step.  Work
 * is replayed from a CUDA graph captured on first use.  Asynchronous.
 * FR_BS32: n_steps attempts of every instance (see FR_BS32); when the call's
 * work is done, every instance's device state is its current (accepted)
 * solution, so fr_get_state, fr_residual and fr_integral see that. */
fr_status fr_rk_step(fr_solver *solver, int n_steps);

/* FR_BS32: the step-control record of instance ``inst`` into out (8 doubles):
 * time t of its current solution, proposed step, step of the next attempt,
 * error norm of the last attempt, 1 if the step being made has had a
 * rejected attempt, accepted attempts, rejected attempts, accepted steps
 * since the last fr_probe_reset.  fr_set_state / fr_set_states restart the
 * instance at t = 0 with the step cfg.dt.  Synchronises.  FR_ERR_INVALID_ARG
 * for other schemes, a null output or an instance out of range. */
fr_status fr_step_control(fr_solver *solver, int inst, double *out8);

/* FR_BS32: move the end time of every instance to t_end (<= 0: none).
 * Instances that had stopped at the old end time continue from there with
 * their proposed step; none goes past the new one.  With it a run reaches a
 * common time in every instance (the end of the transient period, where the
 * observers are reset, Secs. 3.1.2 and 5.2), then goes on.  Synchronises.
 * FR_ERR_INVALID_ARG for other schemes or a NaN time. */
fr_status fr_set_end_time(fr_solver *solver, double t_end);

/* Add an observer at physical point x (dim values) of instance ``inst``; the
 * containing element and reference coordinates are found by Newton's method
 * on the element maps (FP64).  Returns its id in *probe_id.  The pressure is
 * computed from the conserved variables interpolated to x (Sec. 3.1.2). */
fr_status fr_probe_add(fr_solver *solver, int inst, const double *x, int *probe_id);
/* Pressure at the probe after the last completed step (synchronises). */
fr_status fr_probe_pressure(fr_solver *solver, int probe_id, double *p_latest);
/* The most recent pressure samples of one probe since the last reset, oldest
 * first: min(count, 4096, max_n) values into out (host), their number in
 * *n_out (the device keeps a 4096-sample ring per probe), for spectra of the
 * observer signal (Welch PSD, Secs. 3.2, 4.2, 5.2 figures).  Synchronises. */
fr_status fr_probe_history(fr_solver *solver, int probe_id, double *out, int max_n, int *n_out);
/* Checkpoint of everything a step accumulates besides the flow state (which
 * fr_get_state / fr_set_state save): the number of steps in the current
 * averaging window, the wall-force sums of every instance, every probe's
 * FP64 accumulators and sample ring, and (FR_BS32) every instance's
 * step-control record (restored after fr_set_state, it continues the run).  fr_accumulators_size is the number of
 * doubles (-1 for a null solver).  The checkpoint starts with a header: steps
 * in the window, number of probes, number of instances and a fingerprint of
 * the observers (instance and element of each, in order).
 * fr_set_accumulators takes the checkpoint and its length n; it wants a
 * solver with the same instances and the same probes added in the same order
 * and returns FR_ERR_INVALID_ARG, without reading past n, if n is not this
 * solver's fr_accumulators_size or the header disagrees.  States and accumulators
 * restored, the following steps, OASPL and probe histories are bitwise those
 * of an uninterrupted run; the wall-force sums agree to rounding (they are
 * accumulated with atomic additions, whose order varies from run to run).
 * Both synchronise. */
int64_t fr_accumulators_size(const fr_solver *solver);
fr_status fr_get_accumulators(fr_solver *solver, double *out);
fr_status fr_set_accumulators(fr_solver *solver, const double *in, int64_t n);
/* Start a new averaging window: zero all probe and force accumulators. */
fr_status fr_probe_reset(fr_solver *solver);
/* OASPL in dB (Sec. 3.1.2, Eqs. 9-12) over the samples since the last reset:
 * p_RMS of each listed probe (mean_mode 0: p'_i = p_i - running mean up to
 * sample i, the literal reading of Eqs. 11-12; mean_mode 1: p'_i = p_i -
 * window mean), averaged over the probes, OASPL = 20 log10(p_scale p_RMS /
 * p_ref).  Zero variance gives -inf with FR_OK.  Sums are FP64 and
 * compensated. */
fr_status fr_oaspl(fr_solver *solver, const int *probe_ids, int n, double p_ref,
                   double p_scale, int mean_mode, double *oaspl_db);
/* Number of samples in the current window and the sample moments of one
 * probe: out[0] = count, out[1] = mean, out[2] = sum p'^2 (mode 0),
 * out[3] = sum (p - mean)^2 (mode 1). */
fr_status fr_probe_stats(fr_solver *solver, int probe_id, double *out4);

/* Time-mean wall force of instance ``inst`` since the last reset (dim
 * values): sum over wall flux points of w (p n - tau . n) (the force behind
 * C_D, Sec. 3.1.2), averaged over the completed steps (FR_BS32: the
 * instance's accepted steps). */
fr_status fr_forces(fr_solver *solver, int inst, double *mean_force);
/* Time-mean lift and drag coefficients of instance ``inst`` since the last
 * reset (Sec. 3.1.2; the objective of Sec. 5.2 penalises them):
 * C = F . e / (rho_inf |v_inf|^2 a_ref / 2) with F the mean wall force of
 * fr_forces, e the drag direction v_inf / |v_inf| for C_D and the lift
 * direction for C_L (2-D: the drag direction turned by +90 degrees; 3-D: the
 * y axis made orthogonal to the drag direction).  a_ref is the reference
 * length in 2-D (chord) or area in 3-D (chord x span).  FR_ERR_INVALID_ARG
 * for a_ref <= 0, a zero free-stream velocity or (3-D) a free stream along y.
 * Synchronises. */
fr_status fr_force_coefficients(fr_solver *solver, int inst, double a_ref, double *mean_cl,
                                double *mean_cd);

/* Conservation check: FP64 compensated sums over the instance of
 * w_i J_i R_i per variable (zero to round-off on periodic meshes). */
fr_status fr_conservation(fr_solver *solver, int inst, double *sums);
/* Integral of the conserved variables over the instance (FP64), and the
 * number of non-finite state values of that instance in *n_nonfinite. */
fr_status fr_integral(fr_solver *solver, int inst, double *sums, int64_t *n_nonfinite);

/* Allocation-free variant of fr_integral (the paper has no counterpart: it is
 * a service of this library).  Some callers cannot obtain device memory at
 * the point where they want this check: a host application whose memory
 * pool already owns all of the GPU's memory, a monitor that must not grow
 * the solver's workspace, code that may not trigger the implicit device
 * synchronisation an allocation brings.  This entry point allocates nothing
 * and uses no part of the solver's workspace for its reduction: its per-block
 * partial sums live in a fixed device array inside libfr.so (at most
 * 1024 x 11 doubles plus the result, about 90 KB), which every GPU that loads
 * the library holds until the process exits.
 *  - Same inputs and outputs as fr_integral; the sums agree with it to
 *    rounding (the reduction is partitioned differently).
 *  - Limit: the instance may have at most 1024 * 256 * 8 = 2,097,152 solution
 *    points; larger instances get FR_ERR_INVALID_ARG with a message (use
 *    fr_integral for them).
 *  - Every call looks up the array's device address on the current device
 *    (cudaGetSymbolAddress, with that device current), so a device reset
 *    between calls is harmless; make the first call on a device before any
 *    stream capture on it.
 *  - All calls share the one array and it keeps the last call's contents;
 *    each call clears it first.  Calls that overlap on the GPU (other
 *    streams, other threads, other solvers on the same device) race on it:
 *    serialise them.
 *  - Synchronises the solver's stream. */
fr_status fr_integral_static(fr_solver *solver, int inst, double *sums, int64_t *n_nonfinite);

/* Per-instance health of the batch (failure detection inside the time
 * loop; the paper's poll treats a failed evaluation as a rejected candidate,
 * Sec. 2.2).  With cfg.check_every = K > 0, fr_rk_step appends after every
 * K-th step a scan of the state that sets the flag of each instance holding
 * a NaN or Inf; a flag stays set until that instance's state is set again
 * (fr_set_state / fr_set_states).  Instances never interact, so one
 * instance diverging leaves the others' results unchanged.  Synchronises;
 * copies the n_inst flags into ``flags`` (may be NULL), the lowest flagged
 * instance into *first_bad (-1 if none) and returns FR_ERR_NONFINITE if any
 * instance is flagged, else FR_OK. */
fr_status fr_instance_status(fr_solver *solver, int32_t *flags, int *first_bad);

/* Autotuner (a service of this library; the paper has no counterpart).  A
 * solver's stage schedule -- for BR2 batches without mortar faces, one
 * fused kernel per RK stage or a gradient kernel plus a flux kernel -- the
 * register level of its stage kernels (FP32: 0 = the default residency,
 * 1 = one resident CTA fewer per SM and more registers per thread, 2 = one
 * more CTA per SM and fewer registers) and, in
 * FP32, the contraction of the divergence + correction operators (SIMT
 * sum factorisation, or 3xTF32 tensor-core mma products of every element
 * line: FP32-level accuracy, FP32 accumulation) are measured on the
 * solver's own batch: every candidate runs 2 warm-up and 3 timed RK steps
 * (CUDA events) and the fastest is kept.  The
 * result is cached in the JSON file cache_path (NULL: no cache) under a key
 * of the GPU architecture, dimension, degrees, variables, precision,
 * viscous scheme, interface flux, mortar faces and log2 of the solution
 * points.  mode 0: use the cached entry if there is one, else measure and
 * store; 1: always measure and store; 2: use the cached entry if there is
 * one, else keep the current schedule.  Measuring sets every instance to the
 * configuration's free stream and advances it: call fr_tune before
 * fr_set_state (it also clears the probe, force and health accumulators).
 * choice receives "stage=...;regs=...;contract=...;ms=...;source=..." (and, after a
 * measurement, ";candidates=..." with every candidate's ms per step).
 * Synchronises. */
fr_status fr_tune(fr_solver *solver, const char *cache_path, int mode, char *choice, size_t choice_len);
/* The solver's current schedule string (as fr_tune writes it) and its
 * cache key.  Either output may be NULL. */
fr_status fr_schedule(fr_solver *solver, char *schedule, size_t len, char *key, size_t key_len);
/* Host-only cache read: the value stored under key in the JSON file
 * cache_path.  FR_ERR_INVALID_ARG if the file or the key is missing (value
 * is then the empty string). */
fr_status fr_tune_lookup(const char *cache_path, const char *key, char *value, size_t len);

/* Measured arithmetic peak of the current GPU's FMA pipes (a service of this
 * library for roofline fractions of ALU-bound kernels): precision FR_FP64 or
 * FR_FP32; independent FMA chains in every thread of 8 CTAs per SM, 2 flops
 * per FMA, the best of 3 timed launches (CUDA events).  Allocates nothing.
 * Synchronises the device. */
fr_status fr_alu_peak(int precision, double *flops_per_s);

/* Number of kernel launches issued by the last fr_rk_step call. */
int64_t fr_last_launch_count(const fr_solver *solver);

/* Profiling: run n_steps steps without graph replay, with CUDA events on the
 * solver's stream around every launch.  ms[k] = mean duration (ms) of one
 * launch of kind k and count[k] = launches, for k = 0 fused flux/update
 * kernel, 1 BR2 gradient kernel, 2 probe kernel, 3 wall-force kernel,
 * 4 other (5 entries each).  The steps advance the state like fr_rk_step.
 * Synchronises. */
fr_status fr_profile_steps(fr_solver *solver, int n_steps, double *ms, int64_t *count);

const char *fr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FR_H */
