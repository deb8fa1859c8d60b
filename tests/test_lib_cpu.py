"""CPU checks of the C-ABI library (no kernel launches): it loads, exports
every function include/fr.h declares, and its host-side mesh processing
(FP64) agrees with the oracle's and reports bad meshes with error codes."""
import os
import re

import numpy as np
import pytest

from synth import meshes as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fr():
    from paper_2312_14167_gb300 import build, fr as _fr
    if not os.path.exists(os.path.join(ROOT, "paper_2312_14167_gb300", "libfr.so")):
        build.build()
    _fr.lib()
    return _fr


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_function(fr):
    import ctypes
    names = _declared()
    assert len(names) >= 20
    L = ctypes.CDLL(os.path.join(ROOT, "paper_2312_14167_gb300", "libfr.so"))
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert set(fr.EXPORTED) == names


@pytest.mark.parametrize("maker,p", [
    (lambda: M.vortex_mesh(5, jitter=0.2), 3),
    (lambda: M.tgv_mesh(3), 2),
    (lambda: M.cavity_mesh(800), 3),
    (lambda: M.naca_omesh(0.04, 0.3, 0.1, 2.0, 500), 3),
    (lambda: M.tandem_cylinders(2.5, 0.8, 900, 3), 4),
])
def test_host_geometry_matches_oracle(fr, maker, p):
    from oracle.fr import FRDiscretisation
    from oracle.physics import NavierStokes
    mesh = maker()
    lm = fr.Mesh(mesh, p)
    d = FRDiscretisation(mesh, p, NavierStokes(mesh.dim))
    assert lm.n_elem == mesh.n_elem and lm.nsp == d.ref.nsp and lm.nfp == d.ref.nfp
    span = np.ptp(mesh.xyz, axis=0).max()
    assert np.abs(lm.sol_coords() - d.sol_coords()).max() < 1e-13 * span


def test_mesh_errors_are_reported(fr):
    good = M.vortex_mesh(3)
    with pytest.raises(fr.FRError) as e:
        fr.Mesh(good, 5)
    assert e.value.status == 3                       # FR_ERR_UNSUPPORTED
    bad = M.vortex_mesh(3)
    bad.face_tag = bad.face_tag.copy()
    bad.face_tag[0, 0] = 0                           # periodic face marked interior
    with pytest.raises(fr.FRError) as e:
        fr.Mesh(bad, 2)
    assert e.value.status == 2                       # FR_ERR_MESH
    inv = M.vortex_mesh(3)
    inv.elem_vert = inv.elem_vert.copy()
    inv.elem_vert[4] = inv.elem_vert[4][[1, 0, 3, 2]]   # mirrored element: J < 0
    with pytest.raises(fr.FRError) as e:
        fr.Mesh(inv, 2)
    assert e.value.status == 2
    tag = M.vortex_mesh(3)
    tag.face_tag = tag.face_tag.copy()
    tag.face_tag[1, 1] = 9
    with pytest.raises(fr.FRError) as e:
        fr.Mesh(tag, 2)
    assert e.value.status == 1                       # FR_ERR_INVALID_ARG


def test_binding_refuses_arrays_of_the_wrong_shape(fr):
    """The binding checks the mesh arrays' shapes before the C call, which
    reads them by the sizes it is given."""
    import copy
    base = M.naca_omesh(0.04, 0.3, 0.1, 2.0, 500)
    for field, bad in (("xyz", lambda m: m.xyz[:, :1]),
                       ("elem_vert", lambda m: m.elem_vert[:, :3]),
                       ("face_tag", lambda m: m.face_tag[:-1]),
                       ("geo_nodes", lambda m: m.geo_nodes.reshape(-1)[:-2])):
        m = copy.copy(base)
        setattr(m, field, bad(base))
        with pytest.raises(ValueError, match=field):
            fr.Mesh(m, 3)
    assert fr.Mesh(base, 3).n_elem == base.n_elem


def test_solver_needs_a_device_workspace(fr):
    """fr_solver_create refuses a null workspace before touching the GPU."""
    import ctypes as C
    m = fr.Mesh(M.vortex_mesh(3), 2)
    cfg = fr.make_config(2, p_inf=1.0)
    arr = (C.c_void_p * 1)(m.handle)
    assert fr.lib().fr_workspace_bytes(arr, 1, C.byref(cfg)) > 0
    h = C.c_void_p()
    st = fr.lib().fr_solver_create(C.byref(h), arr, 1, C.byref(cfg), None, 0, None)
    assert st == 7                                   # FR_ERR_WORKSPACE
    # an aligned pointer with too few bytes is refused by size, also before any device access
    need = fr.lib().fr_workspace_bytes(arr, 1, C.byref(cfg))
    st = fr.lib().fr_solver_create(C.byref(h), arr, 1, C.byref(cfg), C.c_void_p(256), need - 1, None)
    assert st == 7 and b"too small" in fr.lib().fr_last_error()


def test_adaptive_configuration_is_checked_and_sized(fr):
    """FR_BS32 wants dt > 0 and tolerances that give every variable a positive
    scale (atol_v + rtol > 0); its workspace adds the third RK register and
    the per-element error sums (state size + 8 bytes per element, give or
    take the 256-byte slots of the two buffers)."""
    import ctypes as C
    vm = M.vortex_mesh(4)
    m = fr.Mesh(vm, 2)
    arr = (C.c_void_p * 1)(m.handle)
    base = fr.lib().fr_workspace_bytes(arr, 1, C.byref(fr.make_config(2, p_inf=1.0)))
    good = fr.make_config(2, p_inf=1.0, rk=fr.FR_BS32, dt=0.01, rtol=1e-6, atol=1e-8)
    need = fr.lib().fr_workspace_bytes(arr, 1, C.byref(good))
    n_elem, nsp = vm.elem_vert.shape[0], 9
    extra = n_elem * nsp * 4 * 8 + n_elem * 8
    # (without adaptive steps both buffers still take one 256-byte slot)
    assert extra - 2 * 256 <= need - base <= extra + 2 * 256
    for bad in (dict(dt=0.0, rtol=1e-6, atol=1e-8), dict(dt=0.01, rtol=-1.0, atol=1e-8),
                dict(dt=0.01, rtol=0.0, atol=0.0), dict(dt=0.01, rtol=0.0, atol=[1e-8, 1e-8, 0.0, 1e-8]),
                dict(dt=0.01, rtol=1e-6, atol=-1e-8)):
        cfg = fr.make_config(2, p_inf=1.0, rk=fr.FR_BS32, **bad)
        assert fr.lib().fr_workspace_bytes(arr, 1, C.byref(cfg)) == 0, bad
    # relative tolerance alone is enough; an unknown scheme is refused
    assert fr.lib().fr_workspace_bytes(arr, 1, C.byref(fr.make_config(2, p_inf=1.0, rk=fr.FR_BS32,
                                                                       dt=0.01, rtol=1e-6))) == need
    assert fr.lib().fr_workspace_bytes(arr, 1, C.byref(fr.make_config(2, p_inf=1.0, rk=3))) == 0


@pytest.mark.parametrize("dim", [2, 3])
def test_variable_degree_mesh_host_processing_matches_oracle(fr, dim):
    from oracle.fr_var import VarFRDiscretisation
    from oracle.physics import NavierStokes
    n = (6, 5) if dim == 2 else (3, 3, 2)
    mesh = M.reorient(M.periodic_box(dim, n, (0.0,) * dim, (1.0,) * dim, jitter=0.2), 5)
    ep = M.checker_degrees(mesh, (1, 2, 3, 4), seed=5)
    lm = fr.Mesh(mesh, ep)
    d = VarFRDiscretisation(mesh, ep, NavierStokes(dim))
    assert lm.nsp == 0 and lm.nfp == 0 and lm.n_sp == d.n_sp
    assert np.array_equal(lm.elem_p, ep) and lm.state_shape == (d.n_sp,)
    assert np.abs(lm.sol_coords() - d.sol_coords()).max() < 1e-13
    uni = fr.Mesh(mesh, 3)
    assert uni.n_sp == mesh.n_elem * 4 ** dim and np.all(uni.elem_p == 3)


def test_variable_degree_mesh_errors(fr):
    mesh = M.vortex_mesh(3)
    ep = np.full(mesh.n_elem, 2, dtype=np.int32)
    ep[4] = 5
    with pytest.raises(fr.FRError) as e:
        fr.Mesh(mesh, ep)
    assert e.value.status == 3                       # FR_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        fr.Mesh(mesh, ep[:-1])
    ep[4] = -1
    with pytest.raises(fr.FRError) as e:
        fr.Mesh(mesh, ep)
    assert e.value.status == 3


def test_tuning_cache_lookup_and_fallback(fr, tmp_path):
    """fr_tune_lookup reads the JSON cache fr_tune writes (one "key":
    "value" pair per line); a missing key, a missing file or a line that is
    not a pair gives no schedule (the solver then keeps or measures its own)."""
    import json
    path = tmp_path / "tune.json"
    entries = {"sm_103|dim=2|p=3|V=4|fp32|br2|rusanov|mortar=0|log2sp=23": "stage=split;regs=1;ms=0.8",
               "sm_103|dim=3|p=4|V=5|fp32|br2|rusanov|mortar=0|log2sp=24": "stage=fused;regs=0;ms=2.1"}
    path.write_text(json.dumps(entries, indent=2))
    for k, v in entries.items():
        assert fr.tune_lookup(str(path), k) == v
    assert fr.tune_lookup(str(path), "sm_103|dim=2|p=2|V=4|fp32|br2|rusanov|mortar=0|log2sp=23") is None
    assert fr.tune_lookup(str(tmp_path / "missing.json"), next(iter(entries))) is None
    path.write_text('{\n  not a pair\n  "k": "v"\n}\n')
    assert fr.tune_lookup(str(path), "k") == "v"
    assert fr.tune_lookup(str(path), "not a pair") is None
