"""Multi-rank (N > 1) logic of bench.py on CPU with the gloo backend,
world size 2: each rank works on its own seeded poll, and the whole-job
figures are the slowest rank's time and the sum of the ranks' units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank-dependent work: rank r times (r + 1) ms on (r + 1) * 1000 units
    ms, units = bench.combine_ranks(dist, 1.0 + rank, 1000.0 * (rank + 1), device="cpu")
    # each rank's poll is drawn from its own seed
    from synth import meshes as M
    m = M.airfoil_batch(1, seed=2312 + rank, e_lo=300, e_hi=400)[0]
    out[rank] = (ms, units, float(m.info["m"]), m.n_elem)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_world_size_2_gloo():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0][:2] == out[1][:2] == (2.0, 3000.0)
    assert out[0][2] != out[1][2]          # different candidates per rank


def test_combine_ranks_single_process_passthrough():
    import bench
    assert bench.combine_ranks(None, 3.5, 77) == (3.5, 77)


def test_reference_arm_prints_one_contract_line():
    """``bench.py --impl reference`` (the oracle timed on the host) prints one
    JSON line with the keys of the bench contract, on the default workload."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                       env={**os.environ, "RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    # the oracle ran on every host core (one process each), not the one-core fallback
    import bench
    assert d["cpu_baseline"]["cores"] == bench.host_cores(), d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_bench_taylor_green_diagnostics_match_the_closed_forms():
    """The observer run's kinetic-energy and enstrophy means of the exact
    Taylor-Green field: 1/8 and 3/8 (rho = 1 + O(M^2) at M = 0.1), the
    enstrophy converging with the mesh, and the bench's method bytes per
    update reproducing the scope table's figures (188, 378, 326.4 B)."""
    import numpy as np
    import bench
    from synth import meshes as M, states as S

    def field(n, p):
        m = M.tgv_mesh(n)
        # solution points of the uniform box, in the bench's ordering (xi fastest)
        x1, _, _ = bench._gauss_derivative(p + 1)
        h = 2 * np.pi / n
        lo = m.xyz[m.elem_vert].min(axis=1)
        t = (x1 + 1) / 2 * h
        pts = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1)       # [i][j][k]
        pts = pts.transpose(2, 1, 0, 3).reshape(-1, 3)                 # i fastest
        return S.taylor_green(lo[:, None, :] + pts[None], mach=0.1)

    ek4, en4 = bench.tgv_diagnostics(field(4, 3), 4, 3)
    ek8, en8 = bench.tgv_diagnostics(field(8, 3), 8, 3)
    assert abs(ek8 - 0.125) < 1e-4 and abs(en8 - 0.375) < abs(en4 - 0.375) < 0.05
    saved = bench.W
    try:
        for (w, p), want in ((("airfoil", 3), 188.0), (("tgv", 3), 378.0), (("tandem", 4), 326.4)):
            bench.W = bench.WORKLOADS[w]
            assert abs(bench.method_bytes_per_update(p) - want) < 1e-9
    finally:
        bench.W = saved


def test_stage_traffic_applies_only_to_the_captured_schedule():
    """The bench line's measured stage traffic: the split stage's DRAM bytes
    per update sit a few per cent above the method's minimum of 188 B, and
    no figure is given for a schedule, contraction or workload the capture
    did not cover."""
    import bench
    saved = bench.W
    try:
        bench.W = bench.WORKLOADS["airfoil"]
        rec = bench.NCU_TRAFFIC.get(bench.kernel_source_hash())
        t = bench.stage_traffic("stage=split;regs=0;contract=simt;ms=4.5;source=measured", 1000)
        if rec is None or "grad_bytes_per_elem" not in rec:
            assert t is None
        else:
            assert 188.0 <= t / (1000 * 16) < 200.0
        assert bench.stage_traffic("stage=fused;regs=0;contract=simt;ms=4.7", 1000) is None
        assert bench.stage_traffic("stage=split;regs=0;contract=tc;ms=6.0", 1000) is None
        bench.W = bench.WORKLOADS["tgv"]
        assert bench.stage_traffic("stage=split;regs=2;contract=simt;ms=12.6", 1000) is None
    finally:
        bench.W = saved


def test_oracle_baseline_runs_on_every_core_or_falls_back_to_one(monkeypatch):
    """The oracle's host baseline: one spawned process per host core, each on
    its own element sample (the aggregate counts every process's updates over
    the slowest one's time); if that run fails, one core, with the reason in
    the sample text."""
    import bench
    from synth import meshes as M
    mesh = M.periodic_box(2, (6, 6), (0, 0), (1, 1))
    rec = bench.oracle_baseline(mesh, 8, 1, 2, 1e-4)
    assert rec["cores"] == bench.host_cores() and rec["kind"] == "oracle"
    assert rec["value"] > 0 and rec["per_core_value"] > 0 and rec["seconds"] > 0

    def fail(*a, **k):
        raise RuntimeError("no processes here")

    monkeypatch.setattr(bench, "oracle_all_cores", fail)
    rec = bench.oracle_baseline(mesh, 8, 1, 2, 1e-4)
    assert rec["cores"] == 1 and rec["value"] > 0
    assert "all-core run failed (no processes here)" in rec["sample"]


def test_oracle_all_cores_ends_at_once_when_a_process_dies(monkeypatch):
    """A process that dies without reporting (here: a workload name it does
    not know) ends the all-core run at once with an error, long before its
    time limit."""
    import copy
    import time
    import pytest
    import bench
    from synth import meshes as M
    w = copy.copy(bench.W)
    w.name = "no such workload"
    monkeypatch.setattr(bench, "W", w)
    t0 = time.monotonic()
    with pytest.raises(RuntimeError, match="exit codes"):
        bench.oracle_all_cores(M.periodic_box(2, (4, 4), (0, 0), (1, 1)), 4, 0, 1, 1e-4, limit_s=120.0)
    assert time.monotonic() - t0 < 60.0


def test_parity_summary_flags_a_missed_bound(capsys):
    """The bench's sampled-parity verdict: met when every case is within the
    target and the pointwise forward bound, flagged (and written to stderr)
    when one case misses either."""
    import bench
    ok = {"rel_l2_vs_oracle_exact_input": 8e-6, "max_pointwise_ratio_to_bound": 0.4,
          "pointwise_within_bound": True}
    s = bench.summarise_parity([ok, dict(ok, rel_l2_vs_oracle_exact_input=9e-6)])
    assert s["all_within_target"] and s["all_pointwise_within_bound"]
    assert s["max_rel_l2_vs_oracle_exact_input"] == 9e-6
    assert "misses" not in capsys.readouterr().err
    bad = dict(ok, rel_l2_vs_oracle_exact_input=1.4e-5, max_pointwise_ratio_to_bound=2.8,
               pointwise_within_bound=False)
    s = bench.summarise_parity([ok, bad])
    assert not s["all_within_target"] and not s["all_pointwise_within_bound"]
    assert s["max_pointwise_ratio_to_bound"] == 2.8
    assert "misses a bound" in capsys.readouterr().err
    assert bench.summarise_parity(None) is None


def test_host_cores_respects_a_cgroup_quota(tmp_path):
    """The all-core oracle timing starts one process per core the bench may
    use: the affinity mask, capped by a cgroup CPU quota (rounded up)."""
    import os
    import bench
    aff = len(os.sched_getaffinity(0))
    f = tmp_path / "cpu.max"
    f.write_text("max 100000\n")
    assert bench.host_cores(str(f)) == aff
    f.write_text("150000 100000\n")
    assert bench.host_cores(str(f)) == min(aff, 2)
    f.write_text("50000 100000\n")
    assert bench.host_cores(str(f)) == 1
    assert bench.host_cores(str(tmp_path / "absent")) == aff
