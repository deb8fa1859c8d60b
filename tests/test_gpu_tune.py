"""Autotuner (fr_tune) on the GPU: it measures every candidate schedule
(stage kernels fused or split, register level) on the solver's own batch,
keeps the fastest, caches it, reuses the cache, and every schedule it can
choose gives the oracle's residual."""
import json

import numpy as np
import pytest

from tests import fr_cases as FC

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tune_measures_caches_and_reuses(tmp_path):
    case = FC.airfoil_case(n_inst=2)
    cache = tmp_path / "tune.json"
    sol = FC.lib_solver(case, "fp32")
    choice = sol.tune(str(cache), mode=1)
    print("tuned:", choice)
    parts = dict(kv.split("=", 1) for kv in choice.split(";"))
    assert parts["source"] == "measured" and parts["stage"] in ("fused", "split")
    cands = {c.split("=")[0]: float(c.split("=")[1]) for c in parts["candidates"].split(",")}
    assert set(cands) == {f"{st}/{r}/{c}" for st in ("split", "fused") for r in (0, 1, 2) for c in ("simt", "tc")}
    best = min(cands, key=cands.get)
    assert best == f"{parts['stage']}/{parts['regs']}/{parts['contract']}"
    _, key = sol.schedule()
    stored = json.loads(cache.read_text())
    assert stored[key].startswith(f"stage={parts['stage']};regs={parts['regs']};contract={parts['contract']}")
    # a second solver of the same shape takes the cached choice without measuring
    again = FC.lib_solver(case, "fp32")
    c2 = again.tune(str(cache), mode=0)
    assert "source=cache" in c2 and f"stage={parts['stage']};regs={parts['regs']};contract={parts['contract']}" in c2
    # lookup only with no entry: the default schedule stays
    other = FC.lib_solver(FC.airfoil_case(n_inst=1), "fp32")
    assert "source=default" in other.tune(str(tmp_path / "empty.json"), mode=2)


@pytest.mark.parametrize("contract", ["simt", "tc"])
@pytest.mark.parametrize("stage", ["split", "fused"])
@pytest.mark.parametrize("regs", [0, 1, 2])
def test_every_schedule_matches_the_oracle(tmp_path, stage, regs, contract):
    case = FC.airfoil_case(n_inst=2)
    sol = FC.lib_solver(case, "fp32")
    _, key = sol.schedule()
    cache = tmp_path / "forced.json"
    sched = f"stage={stage};regs={regs};contract={contract}"
    cache.write_text(json.dumps({key: sched + ";ms=1.0"}))
    assert sched in sol.tune(str(cache), mode=2)
    for i in range(2):
        disc = FC.oracle_disc(case, i)
        u = FC.initial_state(case, disc.sol_coords(), i)
        sol.set_state(i, u)
        R32, mag = disc.residual(FC.fp32_input(case, u), magnitude=True)
        err = FC.rel_l2(sol.residual(i), R32)
        bound = 16 * EPS32 * np.linalg.norm(mag) / np.linalg.norm(R32)
        print(f"{sched} airfoil[{i}]: {err:.3e} (bound {bound:.3e})")
        assert err < bound
    sol.rk_step(3)
    assert sol.integral(0)[1] == 0


@pytest.mark.parametrize("name", ["tgv", "tandem"])
@pytest.mark.parametrize("stage", ["split", "fused"])
def test_tensor_core_contraction_3d_matches_the_oracle(tmp_path, name, stage):
    """Hexes (p = 3 Taylor-Green, p = 4 tandem cylinders): the 3xTF32
    tensor-core line contraction against the oracle, within the FP32 bound
    and within 1e-5 of the exact-input residual on the tandem case."""
    case = FC.tgv_case(n=4, p=3) if name == "tgv" else FC.tandem_case(n_inst=1, n_hex=900, n_span=3)
    sol = FC.lib_solver(case, "fp32")
    _, key = sol.schedule()
    cache = tmp_path / "tc.json"
    cache.write_text(json.dumps({key: f"stage={stage};regs=0;contract=tc;ms=1.0"}))
    assert "contract=tc" in sol.tune(str(cache), mode=2)
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    Rg = sol.residual(0)
    R32, mag = disc.residual(FC.fp32_input(case, u), magnitude=True)
    err = FC.rel_l2(Rg, R32)
    total = FC.rel_l2(Rg, disc.residual(u))
    bound = 16 * EPS32 * np.linalg.norm(mag) / np.linalg.norm(R32)
    print(f"{name} {stage} tc: {err:.3e} (bound {bound:.3e}), vs exact input {total:.3e}")
    assert err < bound
    if name == "tandem":
        assert total < 1e-5


def test_alu_peak_measures_both_precisions():
    from paper_2312_14167_gb300 import fr
    p64, p32 = fr.alu_peak(fr.FR_FP64), fr.alu_peak(fr.FR_FP32)
    print(f"FMA peak: FP64 {p64 / 1e12:.2f} TFLOP/s, FP32 {p32 / 1e12:.2f} TFLOP/s")
    assert 0 < p64 < p32 and 1e12 < p32 < 5e14
