#!/usr/bin/env python
"""Throughput benchmark of the FR hot path on one GB300 (or N, weak scaling).

Workload: one MADS poll of NACA 4-digit candidates (Sec. 5 of
arXiv:2312.14167; the batched-airfoil workload): 32 seeded 2-D O-meshes of
8k-40k curved quads, p = 3, compressible Navier-Stokes (BR2) at Re_c = 23000,
M = 0.2, LSRK45, mixed precision (FP32 state/fluxes, FP64 geometry setup and
FP64 probe/force accumulators), one observer per candidate 2 chords below the
trailing edge.  A step is one LSRK45 step of every candidate (5 stages x
(gradient kernel + fused flux/update kernel)) plus the probe and wall-force
sampling kernels, replayed from a CUDA graph.

Metric: solution-point RK-stage updates per second (sum over candidates of
elements x 16 solution points x 5 stages x steps / device time).

Extra keys: the plain FP64 path on the same candidates run one after another
(the comparison the metric names), sampled parity against the FP64 oracle at
full size, the roofline of the dominant kernel, the oracle's own throughput on
the host cores, clocks during the timed region, and an end-to-end figure
through the C ABI with host buffers.

``--impl reference`` times the FP64 oracle (the reference arm: a deliberately
plain CPU program) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import queue
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "sol-pt RK-stage updates/s, batched mixed-prec vs plain FP64 FR, same GB300"
UNIT = "sol-pt RK-stage updates/s"
GAMMA, PR = 1.4, 0.71
STAGES = 5


class Workload:
    """One configuration: dimension, degree, physics, seeded meshes, start."""

    def __init__(self, name, dim, p, re, mach, candidates, desc, make, v_inf, inflow_delta=0.0,
                 start="wall_damped", degrees=None):
        self.name, self.dim, self.p, self.re, self.mach = name, dim, p, re, mach
        self.candidates, self.desc, self.make = candidates, desc, make
        self.v_inf, self.inflow_delta, self.start = v_inf, inflow_delta, start
        # degrees(mesh) -> degree of every element (p is then the highest)
        self.degrees = degrees
        n = p + 1
        self.nsp = n ** dim
        self.nfp = 2 * dim * n ** (dim - 1)
        self.V = dim + 2
        self.MS = dim * dim + 1

    def physics(self):
        return dict(mu=1.0 / self.re, p_inf=1.0 / (GAMMA * self.mach ** 2), v_inf=self.v_inf)

    def elem_degrees(self, mesh):
        if self.degrees is None:
            return np.full(mesh.n_elem, self.p, dtype=np.int32)
        return self.degrees(mesh)

    def sizes(self, p):
        """(solution points, flux points) of one element of degree p."""
        n = p + 1
        return n ** self.dim, 2 * self.dim * n ** (self.dim - 1)


def _airfoils(rank, n):
    from synth import meshes as M
    return M.airfoil_batch(32, seed=2312 + rank, e_lo=8000, e_hi=40000, p_geo=3)[:n]


def _tandems(rank, n):
    from synth import meshes as M
    return M.tandem_batch(16, seed=2312 + rank)[:n] if n == 16 else \
        [M.tandem_cylinders(*a) for a in _tandem_draws(rank)[:n]]


def _tandem_draws(rank):
    rng = np.random.default_rng(2312 + rank)
    out = []
    for _ in range(16):
        s, r, nh = rng.uniform(2.0, 5.0), rng.uniform(0.5, 1.5), int(rng.uniform(60000, 150000))
        out.append((s, r, nh))
    return out


def _sponge(mesh):
    """Variable degree of the airfoil grids (Sec. 5.1, a P0-P3 distribution):
    p = 3 within 4 chords of the mid-chord, p = 2 out to 8, p = 1 out to 12,
    p = 0 in the outer far field."""
    from synth import meshes as M
    return M.sponge_degrees(mesh, (0.5, 0.0), (4.0, 8.0, 12.0), (3, 2, 1, 0))


def _cavity(rank, n):
    from synth import meshes as M
    return [M.cavity_mesh(32000)]


def _tgv(rank, n):
    from synth import meshes as M
    return [M.tgv_mesh(64)]


WORKLOADS = {
    "airfoil": Workload("airfoil", 2, 3, 23000.0, 0.2, 32,
                        "32 NACA 4-digit O-meshes (8k-40k curved quads, seed 2312), p=3, NS BR2, "
                        "Re_c=23000, M=0.2, LSRK45, one probe per candidate", _airfoils, (1.0, 0.0)),
    "airfoil_sponge": Workload("airfoil_sponge", 2, 3, 23000.0, 0.2, 32,
                               "32 NACA 4-digit O-meshes (8k-40k curved quads, seed 2312) with a "
                               "variable degree P0-P3: p=3 within 4c, p=2 to 8c, p=1 to 12c, p=0 beyond (mortar "
                               "coupling), NS BR2, Re_c=23000, M=0.2, LSRK45, one probe per candidate",
                               _airfoils, (1.0, 0.0), degrees=_sponge),
    "tandem": Workload("tandem", 3, 4, 1000.0, 0.2, 16,
                       "16 tandem-cylinder candidates (60k-150k curved hexes, 16 spanwise layers, "
                       "seed 2312), p=4, NS BR2, Re=1000, M=0.2, LSRK45, 16 spanwise probes each",
                       _tandems, (1.0, 0.0, 0.0)),
    "cavity": Workload("cavity", 2, 3, 1500.0, 0.15, 1,
                       "2-D deep-cavity proxy (~32k quads, L/D=0.5), p=3, NS BR2, Re_D=1500, M=0.15, "
                       "tanh inflow, LSRK45, one probe", _cavity, (1.0, 0.0), inflow_delta=0.2),
    "tgv": Workload("tgv", 3, 3, 1600.0, 0.1, 1,
                    "Taylor-Green vortex 64^3 hexes, p=3, NS BR2, Re=1600, M=0.1, LSRK45", _tgv,
                    (0.0, 0.0, 0.0), start="tgv"),
}
W = WORKLOADS["airfoil"]
CANDIDATES = W.candidates     # --candidates: a smaller poll (profiling captures)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the flux and gradient kernels from an ncu capture, per element, valid only
# for the kernel source it was taken on.
NCU_TRAFFIC = {
    # ncu --set full of k_flux<2,4,float,1,0> on the 8-airfoil case (243,854 quads), mean of two
    # launches (profiles/k_flux_airfoil8_full.md), scaled to a launch by the element count
    "9ce1259f965df7a6229c93f4b0d7905bb8e40b0ec59992f643dadead8b30bb73":
        {"flux_bytes_per_elem": ((316.185344e6 + 378.621184e6) / 2 + (151.570944e6 + 153.314560e6) / 2) / 243854},
    # one-pass dram__bytes capture of one split stage on the same case
    # (profiles/traffic_airfoil8_split_stage.md): k_flux<2,4,float,1,0,0> 316.2 MB read
    # + 149.0 MB written, k_grad<2,4,float,0> 249.94 MB + 43.18 MB
    "718c2aecf7009444c359541293d3c384c3fcf704339a068bec575a1ab20458a6":
        {"flux_bytes_per_elem": (316.209920e6 + 148.992000e6) / 243854,
         "grad_bytes_per_elem": (249.94e6 + 43.18e6) / 243854},
}


def stage_traffic(schedule, n_elem):
    """Measured DRAM bytes of one whole RK stage (gradient + flux kernel of
    the split schedule) scaled to ``n_elem`` elements by the element count,
    or None where no capture applies: another kernel source, workload,
    stage schedule or contraction than the one captured."""
    rec = NCU_TRAFFIC.get(kernel_source_hash())
    if not rec or W.name != rec.get("workload", "airfoil"):
        return None
    opts = dict(kv.split("=", 1) for kv in schedule.split(";") if "=" in kv)
    if opts.get("stage") != "split" or opts.get("contract") != "simt":
        return None
    fl, gr = rec.get("flux_bytes_per_elem"), rec.get("grad_bytes_per_elem")
    return (fl + gr) * n_elem if fl and gr else None


# FP64 floating-point operations per solution-point stage update of the plain
# FP64 path (DFMA counted twice, DADD and DMUL once), from an ncu capture of
# its stage kernels on the 8-candidate airfoil case, valid only for the
# kernel source it was taken on
NCU_FP64_FLOPS = {
    # k_grad<2,4,double> 1.9361e8 + k_flux<2,4,double> 3.6875e8 flops per stage over candidate 0
    # (33,800 quads x 16 points), split schedule; profiles/fp64_stage_airfoil8_flops.md
    "9ce1259f965df7a6229c93f4b0d7905bb8e40b0ec59992f643dadead8b30bb73": (1.9361e8 + 3.6875e8) / (33800 * 16),
    "718c2aecf7009444c359541293d3c384c3fcf704339a068bec575a1ab20458a6": (1.93613e8 + 3.68746e8) / (33800 * 16),
}


def kernel_source_hash():
    """sha256 of the kernel source and the build script (its flags)."""
    h = hashlib.sha256()
    for rel in (("csrc", "fr_kernels.cuh"), ("build.py",)):
        with open(os.path.join(ROOT, "paper_2312_14167_gb300", *rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def combine_ranks(dist, ms, units, device="cpu"):
    """Whole-job figures over ranks: the slowest rank's time and the sum of
    the units every rank processed (no data-path collective: candidates are
    independent; only these two scalars cross ranks)."""
    if dist is None:
        return ms, units
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def make_meshes(rank=0):
    return W.make(rank, CANDIDATES)


def cfl_dt(meshes, cfl=0.4):
    """Fixed step from a CFL estimate: smallest corner-edge length over
    (|v| + c) (p+1)^2, the same dt for every candidate."""
    c = np.sqrt(GAMMA * W.physics()["p_inf"])
    hmin = np.inf
    pairs = ((0, 1), (0, 2), (1, 3), (2, 3)) if W.dim == 2 else ((0, 1), (0, 2), (0, 4))
    for m in meshes:
        X = m.xyz[m.elem_vert]
        for a, b in pairs:
            hmin = min(hmin, np.linalg.norm(X[:, a] - X[:, b], axis=1).min())
    return cfl * hmin / ((1.0 + c) * (W.p + 1) ** 2)


def initial_state(x, inst, mesh):
    """Seeded start: free stream with 1 % smooth perturbations, velocity
    damped to zero within about 0.05 of the walls (no impulsive start); the
    Taylor-Green field for that workload."""
    from synth import states as S
    if W.start == "tgv":
        return S.taylor_green(x, mach=W.mach)
    u = S.smooth_perturbed(x, W.dim, W.mach, amp=0.01, seed=7 + inst)
    if "wall_points" in mesh.info:
        u = S.wall_damped(x, mesh.info["wall_points"], 0.05, u)
    return u


def probe_points(mesh):
    if "probes" in mesh.info:
        return list(mesh.info["probes"])
    if "probe" in mesh.info:
        return [mesh.info["probe"]]
    return []


def fp32_input(u):
    """The state the mixed-precision solver computes with for the FP64 state
    u: the FP32 perturbation about the configuration's free stream."""
    from synth import states as S
    ph = W.physics()
    return S.fp32_perturbation_input(u, S.reference_conserved(W.dim, 1.0, ph["v_inf"], ph["p_inf"], GAMMA))


def oracle_phys():
    from oracle.physics import NavierStokes
    ph = W.physics()
    return NavierStokes(W.dim, gamma=GAMMA, mu=ph["mu"], prandtl=PR, viscous=True, rho_inf=1.0,
                        v_inf=ph["v_inf"], p_inf=ph["p_inf"], inflow_delta=W.inflow_delta,
                        inflow_ywall=0.0)


# --------------------------------------------------------------------------
# oracle timing (CPU; reference arm and cpu_baseline)
# --------------------------------------------------------------------------

def oracle_sample_rate(mesh, n_sample, n_steps, dt, seed=0, n_warm=0, barrier=None):
    """Time the FP64 oracle's LSRK45 stages restricted to a sample of
    elements of one candidate (drawn with ``seed``): ``n_warm`` untimed
    steps, then, once ``barrier`` (if given) lets every process through,
    ``n_steps`` timed ones; returns (updates/s, seconds, sample text).
    A variable-degree workload times the variable-degree oracle on the whole
    candidate (it evaluates no element subsets)."""
    if W.degrees is not None:
        return oracle_varp_rate(mesh, max(1, n_steps // 10), dt)
    from oracle.fr import FRDiscretisation
    disc = FRDiscretisation(mesh, W.p, oracle_phys())
    U = initial_state(disc.sol_coords(), 0, mesh)
    rng = np.random.default_rng(seed)
    elems = np.sort(rng.choice(mesh.n_elem, size=min(n_sample, mesh.n_elem), replace=False))
    from oracle.timestep import LSRK45_A, LSRK45_B
    A = [float(a) for a in LSRK45_A]
    B = [float(b) for b in LSRK45_B]

    def lsrk45_steps(n):
        for _ in range(n):
            du = np.zeros((elems.size, W.nsp, W.V))
            for s in range(STAGES):
                R = disc.residual(U, elems)
                du = A[s] * du + dt * R
                U[elems] = U[elems] + B[s] * du

    lsrk45_steps(n_warm)
    if barrier is not None:
        barrier.wait(timeout=600)
    t0 = time.perf_counter()
    lsrk45_steps(n_steps)
    sec = time.perf_counter() - t0
    upd = elems.size * W.nsp * STAGES * n_steps
    return upd / sec, sec, (f"{elems.size} of {mesh.n_elem} elements of candidate 0 "
                            f"(their 2-ring neighbourhood evaluated), {n_steps} LSRK45 steps")


def host_cores(cpu_max="/sys/fs/cgroup/cpu.max"):
    """Host cores this process may run on: its CPU affinity, capped by a
    cgroup CPU quota where one is set (a container may see every core of
    the machine but be given a share of them)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    try:
        with open(cpu_max) as f:
            quota, period = f.read().split()[:2]
        if quota != "max" and float(period) > 0:
            n = min(n, max(1, int(-(-float(quota) // float(period)))))
    except (OSError, ValueError):
        pass
    return n


def _oracle_worker(name, mesh, n_sample, n_warm, n_steps, dt, seed, barrier, results):
    """One host core's share of the all-core oracle timing (a spawned
    process running the single-threaded oracle on its own element sample)."""
    global W
    W = WORKLOADS[name]
    try:
        rate, sec, _ = oracle_sample_rate(mesh, n_sample, n_steps, dt, seed, n_warm, barrier)
        results.put((seed, rate * sec, sec, ""))
    except Exception as ex:  # noqa: BLE001 (reported to the parent)
        barrier.abort()
        results.put((seed, 0.0, 0.0, repr(ex)))


def oracle_all_cores(mesh, n_sample, n_warm, n_steps, dt, limit_s=300.0):
    """The oracle on every host core at once: one spawned process per core,
    each timing ``n_steps`` LSRK45 steps of its own sample of ``n_sample``
    elements, all starting together (a barrier).  Returns (updates/s over all
    cores = all updates / the slowest process's time, median updates/s of one
    process, processes, that time in s).  Raises if any process fails or the
    whole run exceeds ``limit_s``; the processes are joined (or ended) here."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    n = host_cores()
    barrier = ctx.Barrier(n)
    results = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, daemon=True,
                         args=(W.name, mesh, n_sample, n_warm, n_steps, dt, k, barrier, results))
             for k in range(n)]
    for p in procs:
        p.start()
    out = []
    try:
        deadline = time.monotonic() + limit_s
        while len(out) < n:
            try:
                out.append(results.get(timeout=1.0))
            except queue.Empty:
                # a process that died without reporting (or the time limit)
                # ends the run at once instead of at the limit
                dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
                if dead or time.monotonic() > deadline:
                    barrier.abort()
                    raise RuntimeError(f"oracle processes: exit codes {dead}" if dead else
                                       f"oracle processes exceeded {limit_s:.0f} s")
    finally:
        for p in procs:
            p.join(timeout=10)
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)
    errs = [e for *_, e in out if e]
    if errs:
        raise RuntimeError(errs[0])
    upd = sum(u for _, u, _, _ in out)
    sec = max(t for _, _, t, _ in out)
    per = statistics.median(u / t for _, u, t, _ in out)
    return upd / sec, per, n, sec


def oracle_baseline(mesh, n_sample, n_warm, n_steps, dt):
    """The oracle as it stands on the host cores (one-degree workloads):
    every core at once, one process each, or one core if that run fails.
    Returns the ``cpu_baseline`` record (value, unit, cores, kind, sample,
    seconds of the timed region)."""
    try:
        rate, per, n, sec = oracle_all_cores(mesh, n_sample, n_warm, n_steps, dt)
        return {"value": rate, "unit": UNIT, "cores": n, "kind": "oracle",
                "sample": (f"{n} single-threaded processes, one per host core, each {n_sample} of "
                           f"{mesh.n_elem} elements of candidate 0 (its own draw; their 2-ring "
                           f"neighbourhood evaluated), {n_steps} LSRK45 steps after {n_warm} untimed; "
                           "value = all updates / the slowest process's time"),
                "per_core_value": per, "seconds": sec}
    except Exception as ex:  # noqa: BLE001 (fall back to one core, and say so)
        note = f"all-core run failed ({ex}); one core"
    rate, sec, sample = oracle_sample_rate(mesh, n_sample, n_steps, dt, n_warm=n_warm)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"{sample} ({note})",
            "seconds": sec}


def oracle_varp_rate(mesh, n_steps, dt):
    from oracle.fr_var import VarFRDiscretisation
    from oracle.timestep import lsrk45_step
    disc = VarFRDiscretisation(mesh, W.elem_degrees(mesh), oracle_phys())
    U = initial_state(disc.sol_coords(), 0, mesh)
    t0 = time.perf_counter()
    for _ in range(n_steps):
        U = lsrk45_step(disc.residual, U, dt)
    sec = time.perf_counter() - t0
    upd = disc.n_sp * STAGES * n_steps
    return upd / sec, sec, (f"all {mesh.n_elem} elements ({disc.n_sp} solution points) of one "
                            f"candidate, {n_steps} LSRK45 steps of the variable-degree oracle")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    meshes = make_meshes(0)
    dt = cfl_dt(meshes)
    if W.degrees is None:
        m0, steps = meshes[0], args.steps
    else:
        # variable degree: whole-candidate oracle steps of the smallest
        # candidate, at most 3 of them (a few seconds each)
        m0 = min(meshes, key=lambda m: m.n_elem)
        args.steps = steps = max(1, min(args.steps, 3))
    # warm-up steps are untimed, then K timed steps of the bounded sample
    # on every host core (one process each, its own sample)
    if W.degrees is None:
        base = oracle_baseline(m0, 64, max(args.warmup, 1), steps, dt)
    else:
        rate, sec, sample = oracle_sample_rate(m0, 64, steps * 10, dt)
        base = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                "seconds": sec}
    rate, sec = base["value"], base["seconds"]
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_text(), "l2": "n/a (CPU)"},
            "cpu_baseline": base,
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

class Clocks:
    """nvidia-smi sampling during the timed region (a child process we own)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "50", "-i", str(self.dev)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(E, s, kind, p=None):
    """Compulsory DRAM bytes of one launch (the kernel's design, per element):
    flux: state read+write, RK register write (+read in 4 of 5 stages),
    metrics, normals, partner indices, the partner's face state, own and
    partner viscous normal flux, new face state; gradient: state, metrics,
    normals, partner indices, partner face state, viscous normal flux."""
    NSP, NFP = W.sizes(W.p if p is None else p)
    V, MS, D = W.V, W.MS, W.dim
    if kind == "flux":
        per = (NSP * V * s * (3 + 0.8) + NSP * MS * s + NFP * D * s + NFP * 4 + NFP * V * s
               + 2 * NFP * V * s + NFP * V * s)
    elif kind == "stage":
        # fused stage: state r+w, RK register (w + r in 4 of 5 stages), metrics,
        # normals and partner lifting coefficients, partner indices, inbound and
        # outbound face state and gradient flux part
        per = (NSP * V * s * (3 + 0.8) + NSP * MS * s + 2 * NFP * D * s + NFP * 4 + 4 * NFP * V * s)
    else:
        per = NSP * V * s + NSP * MS * s + NFP * D * s + NFP * 4 + NFP * V * s + NFP * V * s
    return per * E


def method_bytes_per_update(p, s=4, s_g=4):
    """The method's minimum DRAM bytes per solution-point stage update with
    fused gathers: read and write the state and one RK register
    (4 V s), the volume metrics ((1 + d^2) s_g), and per flux point (2d/n of
    them per solution point) write the own face state and gradient, read the
    neighbour's ((2V + 2dV) s), and the face normal (d s_g); Euler drops the
    gradient terms.  2-D NS p = 3 FP32: 188 B; 3-D p = 3: 378 B; 3-D p = 4:
    326.4 B."""
    d, V = W.dim, W.V
    n = p + 1
    r_f = 2.0 * d / n
    return 4 * V * s + (1 + d * d) * s_g + r_f * ((2 * V + 2 * d * V) * s + d * s_g)


def sampled_parity(fr, meshes, fms, sol, n_sample=48):
    """Full-size parity on sampled elements of three candidates: FP32 library
    residual vs the FP64 oracle on the FP32-rounded input (within the forward
    error bound) and vs the exact input."""
    from oracle.fr import FRDiscretisation
    out = []
    eps = 2.0 ** -24
    if W.degrees is not None:
        return sampled_parity_varp(meshes, fms, sol)
    for inst in sorted({0, len(fms) // 2, len(fms) - 1}):
        disc = FRDiscretisation(meshes[inst], W.p, oracle_phys())
        u = initial_state(fms[inst].sol_coords(), inst, meshes[inst])
        sol.set_state(inst, u)
        Rg = sol.residual(inst)
        rng = np.random.default_rng(inst)
        el = np.sort(rng.choice(meshes[inst].n_elem, n_sample, replace=False))
        el = np.union1d(el, np.arange(min(8, meshes[inst].n_elem)))    # wall/trailing-edge cells
        u32 = fp32_input(u)
        R32, mag = disc.residual(u32, el, magnitude=True)
        R64 = disc.residual(u, el)
        e_arith = float(np.linalg.norm(Rg[el] - R32) / np.linalg.norm(R32))
        bound = float(16 * eps * np.linalg.norm(mag) / np.linalg.norm(R32))
        e_total = float(np.linalg.norm(Rg[el] - R64) / np.linalg.norm(R64))
        ratio = np.abs(Rg[el] - R32) / np.maximum(16 * eps * mag, 1e-300)
        out.append({"inst": inst, "elements": int(el.size), "rel_l2_vs_oracle_fp32_input": e_arith,
                    "bound": bound, "rel_l2_vs_oracle_exact_input": e_total,
                    "rel_l2_input_rounding_only": float(np.linalg.norm(R32 - R64) / np.linalg.norm(R64)),
                    "within_1e-5": bool(e_total <= 1e-5),
                    "max_pointwise_ratio_to_bound": float(ratio.max()),
                    "pointwise_within_bound": bool(np.all(ratio <= 1.0))})
    return out


def summarise_parity(parity, target=1e-5):
    """One verdict over the sampled parity cases: the worst error against the
    oracle on the exact input beside the mixed-precision target, and whether
    every case met it and every sampled point stayed within the FP32 forward
    bound.  A miss is also written to stderr, so that it is not only a field
    of the line."""
    if not parity:
        return None
    out = {"max_rel_l2_vs_oracle_exact_input": max(c["rel_l2_vs_oracle_exact_input"] for c in parity),
           "target_rel_l2": target,
           "all_within_target": all(c["rel_l2_vs_oracle_exact_input"] <= target for c in parity),
           "max_pointwise_ratio_to_bound": max(c["max_pointwise_ratio_to_bound"] for c in parity),
           "all_pointwise_within_bound": all(c["pointwise_within_bound"] for c in parity)}
    if not (out["all_within_target"] and out["all_pointwise_within_bound"]):
        print("bench: sampled FP32 parity misses a bound: " + json.dumps(out), file=sys.stderr, flush=True)
    return out


def sampled_parity_varp(meshes, fms, sol):
    """Variable degree: the whole residual of the smallest candidate and of
    the last one (FP32 library vs the variable-degree oracle)."""
    from oracle.fr_var import VarFRDiscretisation
    eps = 2.0 ** -24
    out = []
    small = min(range(len(fms)), key=lambda i: meshes[i].n_elem)
    for inst in sorted({small, len(fms) - 1}):
        disc = VarFRDiscretisation(meshes[inst], W.elem_degrees(meshes[inst]), oracle_phys())
        u = initial_state(fms[inst].sol_coords(), inst, meshes[inst])
        sol.set_state(inst, u)
        Rg = sol.residual(inst)
        u32 = fp32_input(u)
        R32, mag = disc.residual(u32, magnitude=True)
        R64 = disc.residual(u)
        ratio = np.abs(Rg - R32) / np.maximum(16 * eps * mag, 1e-300)
        e_total = float(np.linalg.norm(Rg - R64) / np.linalg.norm(R64))
        out.append({"inst": inst, "elements": int(meshes[inst].n_elem), "degrees": "per element",
                    "rel_l2_vs_oracle_fp32_input": float(np.linalg.norm(Rg - R32) / np.linalg.norm(R32)),
                    "bound": float(16 * eps * np.linalg.norm(mag) / np.linalg.norm(R32)),
                    "rel_l2_vs_oracle_exact_input": e_total,
                    "rel_l2_input_rounding_only": float(np.linalg.norm(R32 - R64) / np.linalg.norm(R64)),
                    "within_1e-5": bool(e_total <= 1e-5),
                    "max_pointwise_ratio_to_bound": float(ratio.max()),
                    "pointwise_within_bound": bool(np.all(ratio <= 1.0))})
    return out


def run_gpu(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    meshes = make_meshes(rank)
    dt = cfl_dt(meshes)
    cpu_base = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle runs before the first CUDA call of this process: about
        # 5-10 s of oracle work on each host core
        if W.degrees is None:
            # every host core at once, one process each (spawned: no CUDA here yet)
            cpu_base = oracle_baseline(meshes[0], 256, 2, 20, dt)
        else:
            m_cpu = min(meshes, key=lambda m: m.n_elem)
            rate, sec, sample = oracle_sample_rate(m_cpu, 256, 30, dt)
            cpu_base = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                        "seconds": sec}
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2312_14167_gb300 import fr
    ph = W.physics()
    common = dict(gamma=GAMMA, prandtl=PR, mu=ph["mu"], rho_inf=1.0, v_inf=ph["v_inf"], p_inf=ph["p_inf"],
                  inflow_delta=W.inflow_delta, inflow_ywall=0.0, dt=dt, viscous=True, rk=fr.FR_LSRK45)
    cfg32 = fr.make_config(W.dim, precision=fr.FR_FP32, **common)
    cfg64 = fr.make_config(W.dim, precision=fr.FR_FP64, **common)
    fms = [fr.Mesh(m, W.p if W.degrees is None else W.elem_degrees(m)) for m in meshes]
    E = sum(m.n_elem for m in fms)
    NSPT = sum(m.n_sp for m in fms)                   # solution points of the poll
    by_p = np.bincount(np.concatenate([m.elem_p for m in fms]), minlength=5)
    tune_cache = os.path.join(tempfile.gettempdir(), f"fr_tune_{os.getpid()}.json")
    sol = fr.Solver(fms, cfg32)
    if args.schedule:
        # a fixed schedule (profiling): no measurement, the same launches every run
        _, key = sol.schedule()
        with open(tune_cache, "w") as f:
            json.dump({key: args.schedule}, f)
        schedule = sol.tune(tune_cache, mode=2)
    else:
        schedule = sol.tune(tune_cache, mode=1)   # measured on this batch, before its states are set
    states = [initial_state(m.sol_coords(), i, meshes[i]) for i, m in enumerate(fms)]
    parity = None
    if rank == 0 and not args.no_parity:
        parity = sampled_parity(fr, meshes, fms, sol)
    for i, u in enumerate(states):
        sol.set_state(i, u)
    pids = [[sol.probe_add(i, x) for x in probe_points(meshes[i])] for i in range(len(fms))]
    st = sol.stream
    # warm-up (captures the graph), then the timed steps
    sol.rk_step(args.warmup)
    sol.synchronize()
    sol.probe_reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    e0.record(st)
    sol.rk_step(args.steps)
    e1.record(st)
    e1.synchronize()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    launches = sol.last_launch_count()
    ms, NSPT_all = combine_ranks(dist, ms, NSPT, device="cuda")
    upd_all = NSPT_all * STAGES * args.steps
    value = upd_all / (ms / 1e3)
    # observer results of the timed window
    # an OASPL needs a window of many samples; a short timed run has none
    oaspl = ([sol.oaspl(ids, p_ref=2e-5, p_scale=101325.0 / ph["p_inf"], mean_mode=0)
              for ids in pids[:4] if ids] if args.steps >= 200 else None)
    forces = [list(sol.forces(i)) for i in range(min(2, len(fms)))]
    tot, bad = sol.integral(0)
    # per-kernel times (CUDA events around each launch, no graph)
    n_prof = 3
    kms, kcnt = sol.profile_steps(n_prof)
    kinds = ["flux", "grad", "probe", "force", "other"]
    share = {kinds[k]: float(kms[k] * kcnt[k]) for k in range(5)}
    fused = "stage=fused" in schedule
    dom = max(("flux", "grad"), key=lambda k: share[k])
    kdx = kinds.index(dom)
    dom_model = "stage" if (fused and dom == "flux") else dom
    # one stage's launches of the dominant kind (one per degree group)
    alg = sum(algorithmic_bytes(int(by_p[q]), 4, dom_model, q) for q in range(0, 5) if by_p[q])
    stage_kernel_ms = float(kms[kdx] * kcnt[kdx]) / (n_prof * STAGES)
    achieved = alg / (stage_kernel_ms / 1e3) / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = None
    rec = NCU_TRAFFIC.get(kernel_source_hash())
    if rec and W.name == rec.get("workload", "airfoil"):
        per_elem = rec.get(f"{dom_model}_bytes_per_elem")
        traffic = per_elem * E if per_elem else None
    groups = [q for q in range(0, 5) if by_p[q]]
    kbase = "k_stage" if dom_model == "stage" else f"k_{dom}"
    kname = (f"{kbase}<{W.dim},{W.p + 1},float>" if len(groups) == 1 else
             f"{kbase}<{W.dim},N,float> over the degree groups N = {[q + 1 for q in groups]}, "
             "one launch each per stage")
    # the whole stage at the method's minimum bytes per update: the bench's
    # updates/s times those bytes, against the measured copy bandwidth
    pts = {q: int(by_p[q]) * W.sizes(q)[0] for q in range(0, 5) if by_p[q]}
    b_upd = sum(method_bytes_per_update(q) * n for q, n in pts.items()) / max(sum(pts.values()), 1)
    design_b = sum((algorithmic_bytes(int(by_p[q]), 4, "stage", q) if fused else
                    algorithmic_bytes(int(by_p[q]), 4, "flux", q) + algorithmic_bytes(int(by_p[q]), 4, "grad", q))
                   for q in range(0, 5) if by_p[q]) / max(sum(pts.values()), 1)
    achieved_stage = value / world * b_upd / 1e9
    # measured bytes of one stage over the poll (uniform degree only: the
    # capture is of one degree's kernels)
    traffic_stage = stage_traffic(schedule, E) if len([q for q in range(0, 5) if by_p[q]]) == 1 else None
    roof = {"bound": "hbm", "kernel": "the whole RK stage (every kernel of the step)",
            "achieved": achieved_stage, "peak": peak, "unit": "GB/s", "frac": achieved_stage / peak,
            "traffic": traffic_stage,
            "traffic_bytes_per_update": traffic_stage / NSPT if traffic_stage else None,
            "traffic_how": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one split stage "
                            "(gradient + flux kernel) on 8 of the candidates, scaled to one stage of "
                            "the poll by the element count; null when the kernel source, workload or "
                            "schedule differs from the capture's"),
            "bytes_per_update": b_upd, "design_bytes_per_update": design_b,
            "how": "achieved = (sol-pt stage updates/s per GPU) x the method's minimum bytes per update "
                   "(4 V s + (1 + d^2) s_g + (2d/n)((2V + 2dV) s + d s_g), FP32); peak = measured copy "
                   "bandwidth; design_bytes_per_update = what the chosen schedule's kernels move "
                   "(fused stage kernel, or flux + gradient kernels)",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800",
            "dominant_kernel": {"kernel": kname, "achieved": achieved, "unit": "GB/s", "frac": achieved / peak,
                                "traffic": traffic, "algorithmic_bytes_per_launch": alg,
                                "launch_ms": stage_kernel_ms},
            "stage_ms": float(kms[0] + kms[1]),
            "kernel_ms": {kinds[k]: float(kms[k]) for k in range(5)}}
    del sol
    torch.cuda.empty_cache()

    # end to end through the C ABI: every step uploads the FP64 state of all
    # candidates from pinned host memory, advances one step and reads the state back
    sol = fr.Solver(fms, cfg32)
    sol.tune(tune_cache, mode=0)
    n_all = sum(u.size for u in states)
    pinned = torch.empty(n_all, dtype=torch.float64, pin_memory=True).numpy()
    outs = torch.empty(n_all, dtype=torch.float64, pin_memory=True).numpy()
    pinned[...] = np.concatenate([u.reshape(-1) for u in states])
    n_e2e = max(3, min(args.steps, 10))
    sol.set_states(pinned)
    sol.rk_step(1)
    sol.get_states(out=outs)
    sol.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        sol.set_states(pinned)
        sol.rk_step(1)
        sol.get_states(out=outs)
    sol.synchronize()
    e2e_sec = time.perf_counter() - t0
    e2e_val = NSPT * STAGES * n_e2e / e2e_sec * (NSPT_all / NSPT)
    state_bytes = sum(u.nbytes for u in states)
    del sol
    torch.cuda.empty_cache()

    # adaptive steps (FR_BS32) on the same poll against the fixed-step
    # LSRK45 line above: simulated time per device second (one GPU)
    adaptive = None
    if world == 1 and not args.no_adaptive:
        rtol = 1e-6
        cfg_bs = fr.make_config(W.dim, precision=fr.FR_FP32,
                                **{**common, "rk": fr.FR_BS32, "rtol": rtol,
                                   "atol": adaptive_tolerances(rtol, ph), "check_every": 50})
        n_att = max(20, min(args.steps, 100))
        adaptive = adaptive_run(fr, fms, states, dt, cfg_bs, n_att, 20)
        adaptive.pop("kernel_ms_per_step", None)
        fixed = len(fms) * dt / (ms / args.steps / 1e3)
        adaptive.update({"rtol": rtol, "atol": "rtol x each variable's free-stream scale",
                         "attempts": n_att, "lsrk45_simulated_time_per_device_second": fixed,
                         "speed_vs_fixed_lsrk45": adaptive["simulated_time_per_device_second"] / fixed})

    # the plain single-instance FP64 path, candidates one after another
    n64 = 10
    fp64_sched = []
    t64 = 0.0
    for i, m in enumerate(fms):
        s64 = fr.Solver([m], cfg64)
        sched64 = s64.tune(tune_cache, mode=0)    # one measurement per size bucket
        fp64_sched.append(sched64.split(";source")[0])
        s64.set_state(0, states[i])
        s64.rk_step(1)
        s64.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s64.stream)
        s64.rk_step(n64)
        b.record(s64.stream)
        b.synchronize()
        t64 += a.elapsed_time(b)
        del s64
    fp64_val = NSPT * STAGES * n64 / (t64 / 1e3)
    fp64_alu = None
    alu_peaks = None
    try:
        # FMA-pipe peaks of this GPU (own microbenchmark, CUDA events)
        alu_peaks = {"fp32_gflops": fr.alu_peak(fr.FR_FP32) / 1e9, "source": "fr_alu_peak"}
    except Exception as ex:  # noqa: BLE001 (report, do not fail the bench)
        alu_peaks = {"error": str(ex)}
    try:
        peak64 = fr.alu_peak(fr.FR_FP64)
        alu_peaks["fp64_gflops"] = peak64 / 1e9
        fpu = NCU_FP64_FLOPS.get(kernel_source_hash())
        fp64_alu = {"bound": "alu", "peak_gflops": peak64 / 1e9, "peak_source": "fr_alu_peak (measured FMA chains)",
                    "flops_per_update": fpu,
                    "achieved_gflops": fp64_val * fpu / 1e9 if fpu else None,
                    "frac": fp64_val * fpu / peak64 if fpu else None}
    except Exception as ex:  # noqa: BLE001 (report, do not fail the bench)
        fp64_alu = {"error": str(ex)}
    try:
        os.unlink(tune_cache)
    except OSError:
        pass

    if dist:
        dist.barrier()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_text(),
                           "candidates_per_gpu": len(fms), "elements_per_gpu": E,
                           "sol_pts_per_gpu": NSPT, "p": W.p, "dt": dt,
                           "elements_by_degree": {str(q): int(by_p[q]) for q in range(0, 5) if by_p[q]},
                           "schedule": schedule,
                           "l2": "inputs larger than L2 (FP32 working set %.2f GB > 129 MB), no flush"
                                 % (sum(sol_bytes(int(by_p[q]), q) for q in range(0, 5)) / 1e9)},
                "roofline": roof,
                "cpu_baseline": cpu_base,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                        "d2h_bytes_per_step": state_bytes,
                        "how": "per step: fr_set_states (every candidate, from one pinned FP64 "
                               "host array), fr_rk_step(1), fr_get_states into one pinned FP64 "
                               "host array"},
                "adaptive_steps": adaptive,
                "alu_peaks": alu_peaks,
                "gpu_launches": int(launches),
                "clocks": clocks,
                "fp64_single_instance": {"value": fp64_val, "unit": UNIT,
                                         "ratio_mixed_batched_over_fp64": value / world / fp64_val,
                                         "how": f"FP64 path, one candidate per solver, {n64} steps each, "
                                                "candidates one after another, device time summed",
                                         "roofline": fp64_alu,
                                         "schedules": sorted(set(fp64_sched))},
                "parity": parity,
                "parity_summary": summarise_parity(parity),
                "observers": {"oaspl_db_first4": oaspl,
                              "oaspl_window_samples": args.steps,
                              "mean_force_first2": forces,
                              "state_finite": bool(bad == 0)}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# long-horizon observer runs (--observe N): not a throughput measurement
# --------------------------------------------------------------------------

def _gauss_derivative(n):
    """Gauss-Legendre points and the derivative matrix of the Lagrange basis
    on them (post-processing of sampled states only)."""
    x, w = np.polynomial.legendre.leggauss(n)
    c = np.array([np.prod([x[i] - x[k] for k in range(n) if k != i]) for i in range(n)])
    Dm = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                Dm[i, j] = c[i] / (c[j] * (x[i] - x[j]))
        Dm[i, i] = -Dm[i].sum()
    return x, w, Dm


def tgv_diagnostics(u, n_el, p):
    """Volume means of the kinetic energy rho |v|^2 / 2 and of the enstrophy
    rho |omega|^2 / 2 of a Taylor-Green state on the uniform (2 pi)^3 box of
    n_el^3 hexes (Gauss quadrature, tensor derivative of the velocity)."""
    n = p + 1
    _, w, Dm = _gauss_derivative(n)
    h = 2 * np.pi / n_el
    rho = u[..., 0]
    vel = u[..., 1:4] / rho[..., None]
    W = np.einsum("i,j,k->kji", w, w, w).reshape(-1)            # sp = i + n j + n^2 k
    J = (h / 2) ** 3
    vol = (2 * np.pi) ** 3
    ek = float(np.einsum("es,s->", 0.5 * rho * np.sum(vel * vel, -1), W) * J / vol)
    V = vel.reshape(vel.shape[0], n, n, n, 3)                      # [e][k][j][i][comp]
    dxi = np.einsum("ai,ekjic->ekjac", Dm, V) * (2 / h)            # d/dx
    deta = np.einsum("aj,ekjic->ekaic", Dm, V) * (2 / h)           # d/dy
    dzeta = np.einsum("ak,ekjic->eajic", Dm, V) * (2 / h)          # d/dz
    om = np.stack([deta[..., 2] - dzeta[..., 1], dzeta[..., 0] - dxi[..., 2], dxi[..., 1] - deta[..., 0]], -1)
    om2 = np.sum(om * om, -1).reshape(vel.shape[0], -1)
    ens = float(np.einsum("es,s->", 0.5 * rho * om2, W) * J / vol)
    return ek, ens


def run_observe(args):
    """Long-horizon observer results of one workload, FP32 (mixed, batched)
    and FP64 side by side: OASPL of every candidate over the second half of
    N steps (both mean readings), mean C_L / C_D, and for the Taylor-Green
    workload the kinetic-energy and enstrophy series."""
    import torch
    torch.cuda.set_device(0)
    from paper_2312_14167_gb300 import fr
    meshes = make_meshes(0)
    dt = cfl_dt(meshes)
    ph = W.physics()
    common = dict(gamma=GAMMA, prandtl=PR, mu=ph["mu"], rho_inf=1.0, v_inf=ph["v_inf"], p_inf=ph["p_inf"],
                  inflow_delta=W.inflow_delta, inflow_ywall=0.0, dt=dt, viscous=True, rk=fr.FR_LSRK45,
                  check_every=100)
    fms = [fr.Mesh(m, W.p if W.degrees is None else W.elem_degrees(m)) for m in meshes]
    n = args.observe
    out = {"workload": workload_text(), "steps": n, "dt": dt, "window": "second half"}
    a_ref = 1.0 if W.dim == 2 else float(np.pi)
    for name, prec in (("fp32", fr.FR_FP32), ("fp64", fr.FR_FP64)):
        sol = fr.Solver(fms, fr.make_config(W.dim, precision=prec, **common))
        sol.tune(None, mode=1)
        for i, m in enumerate(fms):
            sol.set_state(i, initial_state(m.sol_coords(), i, meshes[i]))
        pids = [[sol.probe_add(i, x) for x in probe_points(meshes[i])] for i in range(len(fms))]
        series = []
        t0 = time.perf_counter()
        chunk = max(1, n // 20) if W.start == "tgv" else n // 2
        done = 0
        while done < n:
            if W.start == "tgv":
                ek, ens = tgv_diagnostics(sol.get_state(0), round(len(meshes[0].elem_vert) ** (1 / 3)), W.p)
                series.append({"step": done, "t": done * dt, "E_k": ek, "enstrophy": ens})
            k = min(chunk, n - done)
            sol.rk_step(k)
            done += k
            if done == n // 2:
                sol.probe_reset()
        sol.synchronize()
        res = {"seconds": time.perf_counter() - t0, "health": sol.instance_status()[1]}
        if any(pids):
            res["oaspl_db_mode0"] = [sol.oaspl(ids, p_ref=2e-5, p_scale=101325.0 / ph["p_inf"], mean_mode=0)
                                     for ids in pids if ids]
            res["oaspl_db_mode1"] = [sol.oaspl(ids, p_ref=2e-5, p_scale=101325.0 / ph["p_inf"], mean_mode=1)
                                     for ids in pids if ids]
        if "wall_points" in meshes[0].info and W.name != "cavity":
            res["mean_cl_cd"] = [sol.force_coefficients(i, a_ref) for i in range(len(fms))]
        if series:
            ek, ens = tgv_diagnostics(sol.get_state(0), round(len(meshes[0].elem_vert) ** (1 / 3)), W.p)
            series.append({"step": n, "t": n * dt, "E_k": ek, "enstrophy": ens})
            res["series"] = series
        out[name] = res
        del sol
        torch.cuda.empty_cache()
    if "oaspl_db_mode0" in out["fp32"]:
        out["oaspl_fp32_minus_fp64_db"] = [a - b for a, b in zip(out["fp32"]["oaspl_db_mode0"],
                                                               out["fp64"]["oaspl_db_mode0"])]
    print(json.dumps({"observe": out}), flush=True)
    return 0


def adaptive_run(fr, fms, states, dt, cfg, n_timed, warmup, schedule=""):
    """One solver over the poll: `warmup` steps (attempts, for FR_BS32), then
    `n_timed` timed ones (CUDA events on the solver stream): device time,
    simulated time advanced per device second (summed over the candidates)
    and, for adaptive steps, the accepted / rejected attempts and the steps
    taken against the fixed CFL step `dt`."""
    import torch
    n_inst = len(fms)
    adaptive = cfg.rk == fr.FR_BS32
    sol = fr.Solver(fms, cfg)
    if schedule:   # fixed schedule (profiling): no measurement
        _, key = sol.schedule()
        cache = os.path.join(tempfile.gettempdir(), f"fr_tune_adaptive_{os.getpid()}.json")
        with open(cache, "w") as f:
            json.dump({key: schedule}, f)
        sched = sol.tune(cache, mode=2)
        os.unlink(cache)
    else:
        sched = sol.tune(None, mode=1)
    for i, u in enumerate(states):
        sol.set_state(i, u)
    sol.rk_step(warmup)
    sol.synchronize()
    rec0 = [sol.step_control(i) for i in range(n_inst)] if adaptive else None
    st = sol.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    sol.rk_step(n_timed)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    # first instance with a non-finite state (-1: none; scanned every check_every steps)
    res = {"ms": ms, "ms_per_step": ms / n_timed, "schedule": sched.split(";source")[0],
           "first_nonfinite_instance": sol.instance_status()[1]}
    if adaptive:
        rec = [sol.step_control(i) for i in range(n_inst)]
        adv = [r["t"] - a["t"] for r, a in zip(rec, rec0)]
        acc = [r["accepted"] - a["accepted"] for r, a in zip(rec, rec0)]
        rej = [r["rejected"] - a["rejected"] for r, a in zip(rec, rec0)]
        res.update({"accepted": int(sum(acc)), "rejected": int(sum(rej)),
                    "mean_step_over_cfl_dt": float(np.sum(adv) / max(np.sum(acc), 1) / dt),
                    "min_max_h_next_over_cfl_dt": [min(r["h_next"] for r in rec) / dt,
                                                   max(r["h_next"] for r in rec) / dt]})
    else:
        adv = [n_timed * dt] * n_inst
    res["simulated_time_per_device_second"] = float(np.sum(adv) / (ms / 1e3))
    kms, kcnt = sol.profile_steps(3)
    res["kernel_ms_per_step"] = {k: float(kms[j] * kcnt[j] / 3)
                                 for j, k in enumerate(["flux", "grad", "probe", "force", "other"])}
    del sol
    torch.cuda.empty_cache()
    return res


def adaptive_tolerances(rtol, ph):
    """atol at rtol times each conserved variable's free-stream scale."""
    return [rtol * 1.0] + [rtol * 1.0] * W.dim + [rtol * ph["p_inf"] / (GAMMA - 1.0)]


def run_adaptive(args):
    """Adaptive steps (FR_BS32) against fixed LSRK45 steps on one workload,
    FP32 batched: simulated time advanced per second of device time (summed
    over the candidates), the steps the controller takes against the fixed
    CFL step, rejections, and the cost of one attempt against one LSRK45
    step.  Each solver runs `--warmup` steps/attempts, then `--adaptive` timed
    ones."""
    import torch
    torch.cuda.set_device(0)
    from paper_2312_14167_gb300 import fr
    meshes = make_meshes(0)
    dt = cfl_dt(meshes)
    ph = W.physics()
    common = dict(gamma=GAMMA, prandtl=PR, mu=ph["mu"], rho_inf=1.0, v_inf=ph["v_inf"], p_inf=ph["p_inf"],
                  inflow_delta=W.inflow_delta, inflow_ywall=0.0, dt=dt, viscous=True, precision=fr.FR_FP32,
                  check_every=50)
    fms = [fr.Mesh(m, W.p if W.degrees is None else W.elem_degrees(m)) for m in meshes]
    states = [initial_state(m.sol_coords(), i, meshes[i]) for i, m in enumerate(fms)]
    out = {"workload": workload_text(), "cfl_dt": dt, "timed": args.adaptive, "warmup": args.warmup}
    runs = [("lsrk45", dict(rk=fr.FR_LSRK45))]
    for rtol in args.adaptive_rtol:
        runs.append((f"bs32_rtol{rtol:g}", dict(rk=fr.FR_BS32, rtol=rtol, atol=adaptive_tolerances(rtol, ph))))
    for name, kw in runs:
        cfg = fr.make_config(W.dim, **{**common, **kw})
        out[name] = adaptive_run(fr, fms, states, dt, cfg, args.adaptive, args.warmup, args.schedule)
    base = out["lsrk45"]["simulated_time_per_device_second"]
    for name, _ in runs[1:]:
        out[name]["speed_vs_lsrk45"] = out[name]["simulated_time_per_device_second"] / base
    print(json.dumps({"adaptive": out}), flush=True)
    return 0


def sol_bytes(E, p=None):
    s = 4
    NSP, NFP = W.sizes(W.p if p is None else p)
    V = W.V
    return E * (NSP * V * s * 4 + NFP * V * s * 3 + NSP * W.MS * s + NFP * W.dim * s + NFP * 4)


def workload_text():
    if CANDIDATES == W.candidates:
        return W.desc
    return f"{CANDIDATES} of the " + W.desc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adaptive", action="store_true",
                    help="skip the adaptive-steps (FR_BS32) comparison of the default run")
    ap.add_argument("--workload", default="airfoil", choices=sorted(WORKLOADS))
    ap.add_argument("--candidates", type=int, default=0)
    ap.add_argument("--observe", type=int, default=0,
                    help="long-horizon observer run of N steps (OASPL over the second half, FP32 vs FP64)")
    ap.add_argument("--adaptive", type=int, default=0,
                    help="adaptive steps (FR_BS32) against LSRK45: N timed attempts / steps each")
    ap.add_argument("--adaptive-rtol", type=float, nargs="+", default=[1e-6, 1e-4])
    ap.add_argument("--schedule", default="",
                    help="fixed schedule, e.g. 'stage=split;regs=0;contract=simt' (no autotuning)")
    args = ap.parse_args()
    global CANDIDATES, W
    W = WORKLOADS[args.workload]
    CANDIDATES = W.candidates if args.candidates <= 0 else max(1, min(W.candidates, args.candidates))
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.observe > 0:
        return run_observe(args)
    if args.adaptive > 0:
        return run_adaptive(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
