"""Host-side optimisation loop around the GPU FR solver.

The outer level of the paper's two-level parallelism (Sec. 2.2): mesh
adaptive direct search with a minimal positive basis (poll size
n sqrt(mesh size)) or the OrthoMADS maximal basis (poll size
sqrt(mesh size)); the mesh coarsens four-fold after an improving poll and
refines four-fold after a failed one, never beyond its initial size, and the
search ends once the mesh is finer than 1e-6 and the design moved by less
than 1 % over a poll.  All candidates of a poll are evaluated concurrently:
``BatchedPollEvaluator`` advances them as one batch of instances in a single
solver on the GPU.

Also here: the penalised airfoil objective of Sec. 5.2 and a Welch power
spectral density of observer signals (Welch's averaged modified periodogram,
Hann window, 50 % overlap), for the spectra the paper plots.

Nothing here runs on the GPU; the solver calls go through ``fr`` (the C ABI).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

PRIMES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


# --------------------------------------------------------------------------
# poll directions
# --------------------------------------------------------------------------

def poll_size(delta_m: float, n: int, basis: str) -> float:
    """Delta_p of Algorithm 1: n sqrt(Delta_m) (minimal basis) or
    sqrt(Delta_m) (maximal basis)."""
    if basis == "minimal":
        return n * math.sqrt(delta_m)
    if basis == "maximal":
        return math.sqrt(delta_m)
    raise ValueError(basis)


def halton(index: int, dim: int) -> np.ndarray:
    """Radical-inverse (Halton) point number ``index`` in [0,1)^dim."""
    out = np.zeros(dim)
    for d in range(dim):
        b, f, i, r = PRIMES[d], 1.0, index, 0.0
        while i > 0:
            f /= b
            r += f * (i % b)
            i //= b
        out[d] = r
    return out


def householder_basis(t: int, n: int, length: float) -> np.ndarray:
    """Orthogonal integer basis in the manner of OrthoMADS: a Halton point
    mapped to [-1, 1]^n, scaled and rounded to an integer vector q, then the
    columns of H = (q.q) I - 2 q q^T (pairwise orthogonal, all of norm
    q.q), scaled so that their largest entry is about ``length``."""
    u = 2.0 * halton(t, n) - 1.0
    if not np.any(u):
        u[0] = 1.0
    q = np.round(u / np.max(np.abs(u)) * max(1.0, math.sqrt(length)))
    if not np.any(q):
        q[0] = 1.0
    H = float(q @ q) * np.eye(n) - 2.0 * np.outer(q, q)
    scale = length / np.max(np.abs(H))
    return H * scale


def poll_directions(t: int, n: int, delta_m: float, delta_p: float, basis: str) -> np.ndarray:
    """Mesh-scaled poll directions (rows): maximal basis [H, -H] (2n
    directions), minimal basis [H, -sum of the columns of H] (n + 1)."""
    H = householder_basis(t, n, max(delta_p / delta_m, 1.0))
    cols = [H[:, i] for i in range(n)]
    if basis == "maximal":
        dirs = cols + [-c for c in cols]
    elif basis == "minimal":
        dirs = cols + [-np.sum(cols, axis=0)]
    else:
        raise ValueError(basis)
    return np.round(np.asarray(dirs)) * delta_m


# --------------------------------------------------------------------------
# the optimisation loop (Sec. 2.2)
# --------------------------------------------------------------------------

@dataclass
class MadsResult:
    x: np.ndarray
    f: float
    iterations: int           # polls that improved the incumbent
    polls: int
    evaluations: int
    # per poll: (poll number, mesh size the poll used, mesh size after it,
    # incumbent after it, its objective)
    history: list = field(default_factory=list)


def _trial_points(centre, poll_no, mesh_size, basis, lower, upper):
    """The poll's trial designs: centre + each direction of the poll set
    built for this poll (its own Halton point), dropping the null direction
    and anything outside the bounds (an extreme barrier: never evaluated)."""
    n = centre.size
    dirs = poll_directions(poll_no, n, mesh_size, poll_size(mesh_size, n, basis), basis)
    pts = (centre + d for d in dirs if np.any(d))
    return [q for q in pts if np.all(q >= lower) and np.all(q <= upper)]


def _improvement(scores, best):
    """Index of the best strictly improving score, or None."""
    if not scores:
        return None
    i = int(np.argmin(scores))
    return i if scores[i] < best else None


def _settled(mesh_size, x, before, tol_m, tol_x):
    """Stopping rule: the mesh is finer than tol_m and no design variable
    moved by more than tol_x (relative) over the last poll."""
    moved = np.max(np.abs(x - before) / np.maximum(np.abs(before), 1e-300))
    return mesh_size < tol_m and moved < tol_x


def mads(evaluate_poll, x0, delta_m0: float, lower, upper, basis: str = "maximal",
         max_polls: int = 200, tol_m: float = 1e-6, tol_x: float = 0.01) -> MadsResult:
    """Mesh adaptive direct search (Sec. 2.2, Algorithm 1).

    Each poll evaluates the trial designs around the incumbent together
    (``evaluate_poll(list of designs) -> list of objective values``; the
    candidates are independent, so one batched solver run serves a whole
    poll).  The mesh size a poll uses never exceeds the initial one; an
    improving poll moves the incumbent to the best trial and coarsens the
    mesh four-fold, a failed one refines it four-fold.  Trial designs outside
    [lower, upper] are never evaluated."""
    lower, upper = np.asarray(lower, float), np.asarray(upper, float)
    incumbent = np.asarray(x0, float)
    best = float(evaluate_poll([incumbent])[0])
    evaluations, successes = 1, 0
    mesh_size = float(delta_m0)
    record = []
    poll_no = 0
    while poll_no < max_polls:
        poll_no += 1
        used = min(mesh_size, float(delta_m0))
        before = incumbent.copy()
        trials = _trial_points(incumbent, poll_no, used, basis, lower, upper)
        scores = [float(v) for v in evaluate_poll(trials)] if trials else []
        evaluations += len(trials)
        win = _improvement(scores, best)
        if win is None:
            mesh_size = used / 4.0
        else:
            incumbent, best = trials[win], scores[win]
            successes += 1
            mesh_size = used * 4.0
        record.append((poll_no, used, mesh_size, incumbent.copy(), best))
        if _settled(mesh_size, incumbent, before, tol_m, tol_x):
            break
    return MadsResult(x=incumbent, f=best, iterations=successes, polls=poll_no,
                      evaluations=evaluations, history=record)


# --------------------------------------------------------------------------
# objective (Sec. 5.2) and spectra
# --------------------------------------------------------------------------

def penalised_objective(oaspl_db: float, cl: float, cd: float, cl_base: float, cd_base: float,
                        eps1: float = 8000.0, eps2: float = 400000.0) -> float:
    """OASPL + eps1 (C_L - C_L,b)^2, plus eps2 (C_D - C_D,b)^2 only when the
    drag exceeds the baseline's (Sec. 5.2: keep the lift, never raise the
    drag)."""
    f = oaspl_db + eps1 * (cl - cl_base) ** 2
    if cd > cd_base:
        f += eps2 * (cd - cd_base) ** 2
    return f


def welch_psd(x, fs: float, n_windows: int = 6, overlap: float = 0.5):
    """One-sided power spectral density by Welch's method: the signal is cut
    into ``n_windows`` segments overlapping by ``overlap``, each one has its
    mean removed and a periodic Hann window applied, and the periodograms
    (scaled to a density, doubled except at 0 and Nyquist) are averaged.
    The paper's spectra use 6 windows for the cavity (Sec. 3) and 3 for the
    tandem cylinders and the airfoil (Secs. 4 and 5), all at 50 % overlap.
    Returns (frequencies, psd)."""
    x = np.asarray(x, float)
    N = x.size
    nper = int(N / (1 + (n_windows - 1) * (1 - overlap)))
    step = int(round(nper * (1 - overlap)))
    if nper < 2 or step < 1:
        raise ValueError("signal too short")
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(nper) / nper)
    scale = 1.0 / (fs * np.sum(w * w))
    segs = []
    start = 0
    while start + nper <= N:
        seg = x[start:start + nper]
        seg = (seg - seg.mean()) * w
        P = np.abs(np.fft.rfft(seg)) ** 2 * scale
        if nper % 2 == 0:
            P[1:-1] *= 2.0
        else:
            P[1:] *= 2.0
        segs.append(P)
        start += step
    return np.fft.rfftfreq(nper, 1.0 / fs), np.mean(segs, axis=0)


def spl_spectrum(psd, df: float, p_ref: float = 2e-5, p_scale: float = 1.0):
    """Band levels 10 log10(PSD df p_scale^2 / p_ref^2) in dB."""
    return 10.0 * np.log10(np.maximum(np.asarray(psd) * df * p_scale ** 2, 1e-300) / p_ref ** 2)


# --------------------------------------------------------------------------
# one poll = one batched solver
# --------------------------------------------------------------------------

class BatchedPollEvaluator:
    """Evaluates every candidate of a poll together in one FR solver.

    make_mesh(design) -> mesh (a ``synth.meshes.Mesh``-like object) with
    ``info["probe"]`` or ``info["probes"]``; ``start(x, design, mesh) -> u``
    gives the initial state at the solution points; ``objective(oaspl,
    forces, design) -> float`` turns the observer level and the wall forces
    into the objective, ``forces`` being the mean wall force vector, or, with
    ``a_ref`` given, the pair (mean C_L, mean C_D) for that reference length
    or area.  Each call runs ``n_transient`` steps, resets the observers,
    runs ``n_average`` steps and reads the OASPL (running-mean reading of
    Eqs. 11-12).  ``p`` is one degree for every element, or a callable
    mesh -> degree per element (the far-field sponge zones of Sec. 5.1).
    With ``config.check_every > 0`` a candidate whose flow went non-finite
    during the run is flagged by the solver and scores +inf (rejected, like
    an infeasible design).  With adaptive steps (``config.rk == FR_BS32``)
    the horizons are times instead: every candidate advances to
    ``t_transient``, the observers are reset, and every candidate advances
    by ``t_average`` more; a candidate that does not get there within
    ``max_attempts`` attempts per phase (its step collapsed) scores +inf."""

    def __init__(self, make_mesh, p: int, config, n_transient: int, n_average: int, start,
                 objective, p_ref: float = 2e-5, p_scale: float = 1.0, mean_mode: int = 0,
                 a_ref: float | None = None, t_transient: float | None = None,
                 t_average: float | None = None, max_attempts: int = 100000):
        self.make_mesh, self.p, self.cfg = make_mesh, p, config
        self.t_transient, self.t_average, self.max_attempts = t_transient, t_average, max_attempts
        self.n_transient, self.n_average = n_transient, n_average
        self.start, self.objective = start, objective
        self.p_ref, self.p_scale, self.mean_mode = p_ref, p_scale, mean_mode
        self.a_ref = a_ref
        self.last = None

    def __call__(self, designs):
        from . import fr
        if not designs:
            return []
        meshes = [self.make_mesh(d) for d in designs]
        fms = [fr.Mesh(m, self.p(m) if callable(self.p) else self.p) for m in meshes]
        sol = fr.Solver(fms, self.cfg)
        ids = []
        for i, (m, fm) in enumerate(zip(meshes, fms)):
            sol.set_state(i, self.start(fm.sol_coords(), designs[i], m))
            pts = m.info.get("probes", [m.info["probe"]] if "probe" in m.info else [])
            ids.append([sol.probe_add(i, np.asarray(x, float)) for x in pts])
        if self.cfg.rk == fr.FR_BS32:
            if self.t_transient is None or self.t_average is None:
                raise ValueError("adaptive steps need t_transient and t_average")
            ok = sol.advance_to(self.t_transient, max_attempts=self.max_attempts)
            sol.probe_reset()
            ok &= sol.advance_to(self.t_transient + self.t_average, max_attempts=self.max_attempts)
        else:
            sol.rk_step(self.n_transient)
            sol.probe_reset()
            sol.rk_step(self.n_average)
            ok = np.ones(len(designs), dtype=bool)
        failed = sol.instance_status()[0] if self.cfg.check_every > 0 else np.zeros(len(designs), np.int32)
        failed = np.where(ok, failed, 1).astype(np.int32)
        out = []
        for i, d in enumerate(designs):
            if failed[i]:
                out.append(math.inf)
                continue
            level = sol.oaspl(ids[i], self.p_ref, self.p_scale, self.mean_mode)
            forces = sol.forces(i) if self.a_ref is None else sol.force_coefficients(i, self.a_ref)
            out.append(self.objective(level, forces, d))
        self.last = {"designs": list(designs), "objectives": out, "failed": [int(f) for f in failed]}
        sol.close()
        return out
