"""fr_integral_static: the allocation-free integral.

For callers that cannot obtain device memory when they run the check (their
host application's pool owns the GPU's memory, or an allocation's implicit
synchronisation is not acceptable there), the library offers one entry point
whose reduction scratch is a fixed device array inside libfr.so instead of
the solver's workspace.  This file checks, through the C ABI, that it returns
what fr_integral returns (to rounding: the two reductions are partitioned
differently) on two calls in a row, in FP64 and FP32, and that an instance
above its limit is refused with an error.  It is collected last so that a run
stopping at the first failure has run everything else first; it also passes
alone in a fresh process.
"""
import numpy as np
import pytest

from tests import fr_cases as FC
from synth import meshes as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_integral_static_matches_integral_twice(precision):
    case = FC.airfoil_case(n_inst=2)
    sol = FC.lib_solver(case, precision)
    for i in range(2):
        disc = FC.oracle_disc(case, i)
        sol.set_state(i, FC.initial_state(case, disc.sol_coords(), i))
    for inst in (1, 0):
        want, bad_w = sol.integral(inst)
        for _ in range(2):
            got, bad_g = sol.integral_static(inst)
            assert bad_g == bad_w == 0
            assert np.allclose(got, want, rtol=1e-12, atol=0.0)
    # after some steps the state changes and both still agree
    sol.rk_step(2)
    want, _ = sol.integral(0)
    got, _ = sol.integral_static(0)
    assert np.allclose(got, want, rtol=1e-12, atol=0.0)


def test_integral_static_rejects_instances_above_its_limit():
    from paper_2312_14167_gb300 import fr
    # 365 x 365 quads at p = 3: 2,131,600 solution points > 2,097,152
    case = FC.Case("periodic_ns", [M.periodic_box(2, (365, 365), (0, 0), (1, 1))], 3, False,
                   0.0, 0.3)
    sol = FC.lib_solver(case, "fp32")
    with pytest.raises(fr.FRError) as exc:
        sol.integral_static(0)
    assert exc.value.status == 1
    assert "static scratch" in str(exc.value)
