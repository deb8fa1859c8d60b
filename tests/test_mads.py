"""Host optimisation loop (Sec. 2.2, Algorithm 1), the penalised objective
(Sec. 5.2) and the Welch PSD; one GPU test drives a small poll through the
batched solver."""
import math

import numpy as np
import pytest

from paper_2312_14167_gb300 import mads


def test_poll_size_rules():
    assert mads.poll_size(0.25, 3, "minimal") == pytest.approx(1.5)
    assert mads.poll_size(0.25, 3, "maximal") == pytest.approx(0.5)


@pytest.mark.parametrize("basis,count", [("maximal", 8), ("minimal", 5)])
def test_poll_directions_span_positively(basis, count):
    n = 4
    for t in range(1, 20):
        dm = 4.0 ** -(t % 6)
        D = mads.poll_directions(t, n, dm, mads.poll_size(dm, n, basis), basis)
        assert D.shape == (count, n)
        assert np.linalg.matrix_rank(D[:n]) == n
        # on the mesh: every direction is an integer multiple of delta_m
        assert np.allclose(D / dm, np.round(D / dm))
        # positive spanning: every nonzero vector has a direction at an acute angle
        rng = np.random.default_rng(t)
        V = rng.normal(size=(200, n))
        assert np.all(np.max(V @ D.T, axis=1) > 0)


def test_householder_columns_orthogonal():
    for t in (1, 2, 7, 30):
        H = mads.householder_basis(t, 3, 5.0)
        G = H.T @ H
        assert np.allclose(G - np.diag(np.diag(G)), 0.0, atol=1e-9 * np.abs(G).max())


def test_mesh_size_update_and_stopping_follow_algorithm_1():
    """Success multiplies Delta_m by 4 (capped at Delta_m0), failure divides
    it by 4; the loop ends once Delta_m < 1e-6 and the design moved < 1 %."""
    calls = []

    def evaluate(designs):
        calls.append(len(designs))
        # one success (the first poll improves), then only failures
        if len(calls) == 2:
            return [-1.0] + [5.0] * (len(designs) - 1)
        return [5.0] * len(designs) if len(calls) > 1 else [0.0]

    res = mads.mads(evaluate, [1.0, 2.0], 0.25, [-10, -10], [10, 10], basis="maximal")
    used = [h[1] for h in res.history]
    after = [h[2] for h in res.history]
    assert used[0] == 0.25 and after[0] == 1.0      # success: x 4
    assert used[1] == 0.25                          # capped at the initial mesh size
    for u, a in zip(used[1:], after[1:]):
        assert a == pytest.approx(u / 4.0)          # failures: / 4
    assert after[-1] < 1e-6 and after[-2] >= 1e-6
    assert res.iterations == 1 and res.f == -1.0


def test_mads_minimises_a_smooth_function_in_bounds():
    target = np.array([0.3, -1.2, 2.0])

    def evaluate(designs):
        return [float(np.sum((np.asarray(d) - target) ** 2)) for d in designs]

    for basis in ("maximal", "minimal"):
        res = mads.mads(evaluate, [1.0, 1.0, 1.0], 1.0, [-5] * 3, [5] * 3, basis=basis, max_polls=400)
        assert np.linalg.norm(res.x - target) < 5e-3
        assert res.evaluations > res.polls


def test_candidates_outside_bounds_are_not_evaluated():
    seen = []

    def evaluate(designs):
        seen.extend(designs)
        return [abs(d[0]) for d in designs]

    mads.mads(evaluate, [0.9], 1.0, [0.0], [1.0], basis="maximal", max_polls=10)
    assert all(0.0 <= d[0] <= 1.0 for d in seen)


def test_penalised_objective_closed_forms():
    assert mads.penalised_objective(110.0, 0.65, 0.05, 0.65, 0.06) == 110.0
    assert mads.penalised_objective(110.0, 0.66, 0.05, 0.65, 0.06) == pytest.approx(110.0 + 8000 * 1e-4)
    assert mads.penalised_objective(110.0, 0.65, 0.061, 0.65, 0.06) == pytest.approx(110.0 + 400000 * 1e-6)


def test_welch_psd_matches_library_and_parseval():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    fs = 200.0
    t = np.arange(7000) / fs
    x = 0.7 * np.sin(2 * np.pi * 12.5 * t) + 0.2 * rng.normal(size=t.size) + 3.0
    for k in (3, 6):
        f, P = mads.welch_psd(x, fs, n_windows=k)
        nper = int(x.size / (1 + (k - 1) * 0.5))
        f2, P2 = signal.welch(x, fs, window="hann", nperseg=nper, noverlap=nper - int(round(nper / 2)),
                              detrend="constant", scaling="density")
        assert np.allclose(f, f2) and np.allclose(P, P2, rtol=1e-10, atol=1e-14)
    # the spectral peak sits at the tone
    assert abs(f[np.argmax(P)] - 12.5) < f[1]


@pytest.mark.gpu
def test_batched_poll_evaluator_runs_a_poll_on_the_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_14167_gb300 import fr
    from synth import meshes as M, states as S
    from tests import fr_cases as FC

    def make_mesh(d):
        return M.naca_omesh(d[0], 0.4, d[1], 3.0, 300)

    probe = M.naca_omesh(0.02, 0.4, 0.12, 3.0, 300)
    dt = FC.cfl_dt([probe], 0.2, 3)
    cfg = fr.make_config(2, mu=1 / 23000, v_inf=(1.0, 0.0), p_inf=1 / (1.4 * 0.04), dt=dt,
                         viscous=True, precision=fr.FR_FP32)

    def start(x, d, m):
        return S.wall_damped(x, m.info["wall_points"], 0.05, S.smooth_perturbed(x, 2, 0.2, amp=0.01))

    def objective(level, force, d):
        cd, cl = force[0] / 0.5, force[1] / 0.5
        return mads.penalised_objective(level, cl, cd, 0.3, 0.05)

    ev = mads.BatchedPollEvaluator(make_mesh, 3, cfg, 5, 20, start, objective,
                                   p_scale=101325 * 1.4 * 0.04)
    vals = ev([np.array([0.02, 0.12]), np.array([0.03, 0.10]), np.array([0.01, 0.14])])
    assert len(vals) == 3 and all(np.isfinite(vals))
    # the same poll on grids with a lower-degree far field (a degree per element)
    ev2 = mads.BatchedPollEvaluator(make_mesh, lambda m: M.sponge_degrees(m, (0.5, 0.0), (2.0, 6.0), (3, 2, 1)),
                                    cfg, 5, 20, start, objective, p_scale=101325 * 1.4 * 0.04)
    vals2 = ev2([np.array([0.02, 0.12]), np.array([0.03, 0.10])])
    assert len(vals2) == 2 and all(np.isfinite(vals2))
    # coefficients from the library (chord 1) and the in-loop health scan: the
    # objective sees (C_L, C_D); a candidate started from a NaN is rejected
    cfg.check_every = 5

    def objective_c(level, coeffs, d):
        return mads.penalised_objective(level, coeffs[0], coeffs[1], 0.3, 0.05)

    def start_bad(x, d, m):
        u = start(x, d, m)
        if d[0] > 0.025:
            u[0, 0, 0] = np.nan
        return u

    ev3 = mads.BatchedPollEvaluator(make_mesh, 3, cfg, 5, 20, start_bad, objective_c,
                                    p_scale=101325 * 1.4 * 0.04, a_ref=1.0)
    vals3 = ev3([np.array([0.02, 0.12]), np.array([0.03, 0.10])])
    assert np.isfinite(vals3[0]) and vals3[0] == pytest.approx(vals[0], rel=1e-12)
    assert vals3[1] == math.inf and ev3.last["failed"] == [0, 1]


@pytest.mark.gpu
def test_batched_poll_evaluator_with_adaptive_steps():
    """Adaptive steps: every candidate advances to the end of the transient
    period (a common time), the observers are reset, every candidate advances
    through the averaging window; a candidate started from a NaN never gets
    there (its step collapses) and scores +inf, and the healthy candidate's
    objective does not depend on the other one."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_14167_gb300 import fr
    from synth import meshes as M, states as S
    from tests import fr_cases as FC

    def make_mesh(d):
        return M.naca_omesh(d[0], 0.4, d[1], 3.0, 300)

    dt = FC.cfl_dt([make_mesh((0.02, 0.12))], 0.2, 3)
    p_inf = 1 / (1.4 * 0.04)
    cfg = fr.make_config(2, mu=1 / 23000, v_inf=(1.0, 0.0), p_inf=p_inf, dt=dt, viscous=True,
                         precision=fr.FR_FP32, rk=fr.FR_BS32, rtol=1e-6,
                         atol=[1e-6, 1e-6, 1e-6, 1e-6 * p_inf / 0.4], check_every=5)

    def start(x, d, m):
        return S.wall_damped(x, m.info["wall_points"], 0.05, S.smooth_perturbed(x, 2, 0.2, amp=0.01))

    def start_bad(x, d, m):
        u = start(x, d, m)
        if d[0] > 0.025:
            u[0, 0, 0] = np.nan
        return u

    def objective(level, coeffs, d):
        return mads.penalised_objective(level, coeffs[0], coeffs[1], 0.3, 0.05)

    kw = dict(p_scale=101325 * 1.4 * 0.04, a_ref=1.0, t_transient=5 * dt, t_average=20 * dt,
              max_attempts=300)
    ev = mads.BatchedPollEvaluator(make_mesh, 3, cfg, 0, 0, start, objective, **kw)
    vals = ev([np.array([0.02, 0.12]), np.array([0.01, 0.14])])
    assert all(np.isfinite(vals)) and ev.last["failed"] == [0, 0]
    ev2 = mads.BatchedPollEvaluator(make_mesh, 3, cfg, 0, 0, start_bad, objective, **kw)
    vals2 = ev2([np.array([0.02, 0.12]), np.array([0.03, 0.10])])
    assert vals2[0] == vals[0]
    assert vals2[1] == math.inf and ev2.last["failed"] == [0, 1]
