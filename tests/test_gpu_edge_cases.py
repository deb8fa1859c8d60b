"""Edge cases of the CUDA path, against the oracle where there is a result:
ragged element tiles for every degree and dimension, single-element
periodic meshes (an element that is its own neighbour on every face), an
element whose every face is a boundary, p = 1; empty / no-op calls and
argument errors; non-finite detection; checkpoint and resume through
fr_get_state / fr_set_state bitwise equal to an uninterrupted run."""
import numpy as np
import pytest

from tests import fr_cases as FC
from synth import meshes as M, states as S
from oracle import timestep as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(mesh, p, visc=True):
    v_inf = (1.0, 0.0) if mesh.dim == 2 else (1.0, 0.0, 0.0)
    return FC.Case("edge", [mesh], p, visc, 0.01 if visc else 0.0, 0.3, dt=1e-3, v_inf=v_inf)


def _parity(case, tol=1e-12):
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = S.smooth_perturbed(disc.sol_coords(), case.dim, case.mach, amp=0.05, seed=3)
    sol.set_state(0, u)
    err = FC.rel_l2(sol.residual(0), disc.residual(u))
    assert err < tol, err
    sol.rk_step(2)
    ur = u
    for _ in range(2):
        ur = T.lsrk45_step(disc.residual, ur, case.dt)
    assert FC.rel_l2(sol.get_state(0), ur) < tol


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_ragged_tiles_2d(p):
    """Element counts that leave a partial last tile (tiles hold 256/(p+1)^2 elements)."""
    ne = 256 // (p + 1) ** 2
    nx = ne + 1
    _parity(_case(M.periodic_box(2, (nx, 1), (0, 0), (1.0 * nx, 1.0), jitter=0.0), p))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_ragged_tiles_3d(p):
    _parity(_case(M.periodic_box(3, (3, 2, 1), (0, 0, 0), (1.5, 1.0, 0.7), jitter=0.0), p))


@pytest.mark.parametrize("dim", [2, 3])
def test_single_element_periodic_in_every_direction(dim):
    box = M.periodic_box(dim, (1,) * dim, (0,) * dim, (1.0,) * dim)
    _parity(_case(box, 3))


def test_element_with_every_face_on_a_boundary():
    m = M.periodic_box(2, (1, 1), (0, 0), (1, 1))
    m.face_tag = m.face_tag.copy()
    m.face_tag[0] = [M.TAG_FARFIELD, M.TAG_OUTFLOW, M.TAG_WALL, M.TAG_FARFIELD]
    _parity(_case(m, 3))


def test_no_op_and_argument_errors():
    from paper_2312_14167_gb300 import fr
    case = _case(M.vortex_mesh(3), 2)
    sol = FC.lib_solver(case, "fp64")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    sol.set_state(0, u)
    sol.rk_step(0)                                   # no steps: state unchanged
    assert np.array_equal(sol.get_state(0), u)
    buf = np.empty_like(u)                           # caller-provided output, written in place
    assert sol.get_state(0, out=buf) is buf and np.array_equal(buf, u)
    with pytest.raises(ValueError):
        sol.get_state(0, out=np.empty(u.shape, dtype=np.float32))
    # no instance 1: the binding's list index refuses it, and so does the C ABI
    with pytest.raises(IndexError):
        sol.set_state(1, u)
    assert fr.lib().fr_set_state(sol.handle, 1, fr._dptr(u)) == 1
    assert fr.lib().fr_set_state(sol.handle, -1, fr._dptr(u)) == 1
    with pytest.raises(fr.FRError) as e:
        sol.probe_add(0, np.array([100.0, 100.0]))   # outside the mesh
    assert e.value.status == 1
    with pytest.raises(fr.FRError):
        sol.oaspl([0])                               # no probe 0 yet
    with pytest.raises(ValueError):
        sol.set_state(0, u[:-1])                     # wrong shape, refused by the binding
    empty = M.vortex_mesh(3)
    empty.elem_vert = empty.elem_vert[:0]
    empty.face_tag = empty.face_tag[:0]
    with pytest.raises(fr.FRError) as e:
        fr.Mesh(empty, 2)                            # an empty mesh is refused
    assert e.value.status == 1


def test_non_finite_state_is_reported():
    case = _case(M.vortex_mesh(4), 2)
    sol = FC.lib_solver(case, "fp32")
    disc = FC.oracle_disc(case)
    u = FC.initial_state(case, disc.sol_coords())
    u[5, 3, 1] = np.nan
    u[7, 0, 0] = np.inf
    sol.set_state(0, u)
    _, bad = sol.integral(0)
    assert bad == 2
    _, bad2 = sol.integral_static(0)
    assert bad2 == 2


@pytest.mark.parametrize("rk", ["lsrk45", "rk4"])
def test_checkpoint_resume_is_bitwise_equal(rk):
    import dataclasses
    case = dataclasses.replace(FC.airfoil_case(n_inst=2), rk=rk)
    full = FC.lib_solver(case, "fp32")
    us = []
    for i in range(2):
        disc = FC.oracle_disc(case, i)
        u = FC.initial_state(case, disc.sol_coords(), i)
        full.set_state(i, u)
        us.append(u)
    full.rk_step(6)
    first = FC.lib_solver(case, "fp32")
    for i in range(2):
        first.set_state(i, us[i])
    first.rk_step(3)
    ckpt = [first.get_state(i) for i in range(2)]    # FP64 copies of the FP32 state: exact
    resumed = FC.lib_solver(case, "fp32")
    for i in range(2):
        resumed.set_state(i, ckpt[i])
    resumed.rk_step(3)
    for i in range(2):
        assert np.array_equal(resumed.get_state(i), full.get_state(i))


def test_checkpoint_resume_with_observers_is_bitwise_equal():
    """States (fr_get_state) and accumulators (fr_get_accumulators) saved
    mid-window and restored into a fresh solver with the same probes: the
    state, OASPL and probe history after the remaining steps are bitwise
    those of the uninterrupted run; the mean wall force agrees to rounding
    (its sums use atomic additions, whose order varies between runs)."""
    from paper_2312_14167_gb300 import fr
    case = FC.airfoil_case(n_inst=2)
    us = [FC.initial_state(case, FC.oracle_disc(case, i).sol_coords(), i) for i in range(2)]

    def fresh():
        sol = FC.lib_solver(case, "fp32")
        for i in range(2):
            sol.set_state(i, us[i])
        ids = [sol.probe_add(i, np.asarray(case.meshes[i].info["probe"], float)) for i in range(2)]
        sol.probe_reset()
        return sol, ids

    full, ids = fresh()
    full.rk_step(6)
    first, ids1 = fresh()
    first.rk_step(3)
    states = [first.get_state(i) for i in range(2)]
    acc = first.get_accumulators()
    assert acc.size == fr.lib().fr_accumulators_size(first.handle) and acc[0] == 3 and acc[1] == 2
    assert acc[2] == 2
    resumed = FC.lib_solver(case, "fp32")
    ids2 = [resumed.probe_add(i, np.asarray(case.meshes[i].info["probe"], float)) for i in range(2)]
    for i in range(2):
        resumed.set_state(i, states[i])
    resumed.set_accumulators(acc)
    resumed.rk_step(3)
    assert resumed.oaspl(ids2) == full.oaspl(ids)
    for i in range(2):
        assert np.array_equal(resumed.get_state(i), full.get_state(i))
        assert np.allclose(resumed.forces(i), full.forces(i), rtol=1e-12, atol=0.0)
        assert np.array_equal(resumed.probe_history(ids2[i]), full.probe_history(ids[i]))
    lone = FC.lib_solver(case, "fp32")                 # no probes: the checkpoint does not fit
    assert fr.lib().fr_set_accumulators(lone.handle, fr._dptr(acc), acc.size) == 1
    with pytest.raises(ValueError):
        lone.set_accumulators(acc)
    # same probe count, other locations: the fingerprint refuses it
    other = FC.lib_solver(case, "fp32")
    for i in range(2):
        other.probe_add(i, np.asarray(case.meshes[i].info["probe"], float) + np.array([0.3, 0.2]))
    assert fr.lib().fr_set_accumulators(other.handle, fr._dptr(acc), acc.size) == 1
    # a solver with one instance fewer: the size check refuses it before any read
    single = fr.Solver([fr.Mesh(case.meshes[0], case.p)], FC.lib_config(case, "fp32"))
    single.probe_add(0, np.asarray(case.meshes[0].info["probe"], float))
    single.probe_add(0, np.asarray(case.meshes[0].info["probe"], float))
    assert fr.lib().fr_set_accumulators(single.handle, fr._dptr(acc), acc.size) == 1


def test_non_finite_instance_is_flagged_inside_the_time_loop():
    """A NaN planted (on the host) in one instance of a batch: the scan that
    fr_rk_step appends every check_every steps flags that instance alone,
    and the other instances advance exactly as they do alone."""
    from paper_2312_14167_gb300 import fr
    case = FC.airfoil_case(n_inst=3)
    cfg = FC.lib_config(case, "fp32")
    cfg.check_every = 2
    ms = [fr.Mesh(m, case.p) for m in case.meshes]
    sol = fr.Solver(ms, cfg)
    us = [FC.initial_state(case, ms[i].sol_coords(), i) for i in range(3)]
    bad = us[1].copy()
    bad[5, 3, 0] = np.nan
    for i in range(3):
        sol.set_state(i, bad if i == 1 else us[i])
    flags, first = sol.instance_status()
    assert first == -1 and not flags.any()          # no scan has run yet
    sol.rk_step(4)
    flags, first = sol.instance_status()
    assert first == 1 and list(flags) == [0, 1, 0]
    assert sol.last_launch_count() > 0
    for i in (0, 2):
        solo = fr.Solver([ms[i]], cfg)
        solo.set_state(0, us[i])
        solo.rk_step(4)
        assert np.array_equal(sol.get_state(i), solo.get_state(0))
    # setting the instance's state again clears its flag
    sol.set_state(1, us[1])
    assert sol.instance_status()[1] == -1
    sol.rk_step(2)
    assert sol.instance_status()[1] == -1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("degrees", [(3, 3, 3), (2, 3, 2)])
def test_batch_transfers_equal_per_instance_transfers(precision, degrees):
    """fr_set_states / fr_get_states move the whole batch through one FP64
    staging copy each way when no instance spans several degree groups (one
    group, or uniform instances of different degrees, whose conversions run
    over runs of consecutive instances): bitwise the per-instance calls, and
    the residuals and steps that follow are bitwise the same too."""
    from paper_2312_14167_gb300 import fr
    ms = M.airfoil_batch(3, seed=11, e_lo=200, e_hi=320, p_geo=3)
    case = FC.airfoil_case(n_inst=1, e_lo=200, e_hi=201)
    cfg = FC.lib_config(case, precision)

    def solver():
        return fr.Solver([fr.Mesh(m, p) for m, p in zip(ms, degrees)], cfg)
    a, b = solver(), solver()
    us = [S.wall_damped(a.meshes[i].sol_coords(), ms[i].info["wall_points"], 0.05,
                        S.smooth_perturbed(a.meshes[i].sol_coords(), 2, 0.2, amp=0.05, seed=i))
          for i in range(3)]
    for i, u in enumerate(us):
        a.set_state(i, u)
    b.set_states(np.concatenate([u.reshape(-1) for u in us]))
    flat = b.get_states()
    assert np.array_equal(flat, np.concatenate([a.get_state(i).reshape(-1) for i in range(3)]))
    for i in range(3):
        assert np.array_equal(a.get_state(i), b.get_state(i))
        assert np.array_equal(a.residual(i), b.residual(i))
    a.rk_step(2)
    b.rk_step(2)
    assert np.array_equal(b.get_states(), np.concatenate([a.get_state(i).reshape(-1) for i in range(3)]))
