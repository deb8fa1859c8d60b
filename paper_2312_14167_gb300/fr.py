"""Thin Python binding of libfr.so (include/fr.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; PyTorch
supplies the device workspace (a uint8 tensor) and the CUDA stream.  There is
no CPU fallback: importing this module fails loudly when libfr.so is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libfr.so")

FR_OK = 0
FR_TAG_INTERIOR, FR_TAG_PERIODIC, FR_TAG_WALL = 0, 1, 2
FR_TAG_FARFIELD, FR_TAG_INFLOW, FR_TAG_OUTFLOW = 3, 4, 5
FR_RK4, FR_LSRK45, FR_BS32 = 0, 1, 2
FR_FP64, FR_FP32 = 0, 1
FR_FLUX_RUSANOV, FR_FLUX_ROE = 0, 1
FR_VISC_BR2, FR_VISC_LDG = 0, 1

STATUS = {0: "FR_OK", 1: "FR_ERR_INVALID_ARG", 2: "FR_ERR_MESH", 3: "FR_ERR_UNSUPPORTED",
          4: "FR_ERR_CUDA", 5: "FR_ERR_NONFINITE", 6: "FR_ERR_TIMEOUT", 7: "FR_ERR_WORKSPACE"}

EXPORTED = ["fr_mesh_create", "fr_mesh_create_varp", "fr_mesh_degrees", "fr_mesh_destroy",
            "fr_mesh_info", "fr_mesh_sol_coords",
            "fr_workspace_bytes", "fr_solver_create", "fr_solver_destroy", "fr_set_state",
            "fr_set_states", "fr_get_states", "fr_accumulators_size", "fr_get_accumulators",
            "fr_set_accumulators",
            "fr_get_state", "fr_residual", "fr_rk_step", "fr_probe_add", "fr_probe_pressure",
            "fr_probe_history",
            "fr_probe_reset", "fr_oaspl", "fr_probe_stats", "fr_forces", "fr_conservation",
            "fr_integral", "fr_integral_static", "fr_last_launch_count", "fr_profile_steps",
            "fr_instance_status", "fr_force_coefficients", "fr_tune", "fr_schedule", "fr_tune_lookup",
            "fr_alu_peak", "fr_step_control", "fr_set_end_time",
            "fr_last_error"]


class FRError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("gamma", C.c_double), ("prandtl", C.c_double), ("mu", C.c_double),
                ("rho_inf", C.c_double), ("v_inf", C.c_double * 3), ("p_inf", C.c_double),
                ("inflow_delta", C.c_double), ("inflow_ywall", C.c_double),
                ("br2_eta", C.c_double), ("dt", C.c_double), ("viscous", C.c_int),
                ("rk", C.c_int), ("precision", C.c_int), ("flux", C.c_int),
                ("viscous_scheme", C.c_int), ("check_every", C.c_int), ("ldg_beta", C.c_double),
                ("ldg_tau", C.c_double), ("flux_reference", C.c_int), ("reserved", C.c_int),
                ("t_end", C.c_double), ("dt_max", C.c_double), ("rtol", C.c_double),
                ("atol", C.c_double * 5)]


def make_config(dim, gamma=1.4, prandtl=0.71, mu=0.0, rho_inf=1.0, v_inf=None, p_inf=1.0,
                inflow_delta=0.0, inflow_ywall=0.0, br2_eta=0.0, dt=1e-3, viscous=False,
                rk=FR_LSRK45, precision=FR_FP64, flux=FR_FLUX_RUSANOV,
                viscous_scheme=FR_VISC_BR2, ldg_beta=0.5, ldg_tau=0.1, check_every=0,
                flux_reference=0, t_end=0.0, dt_max=0.0, rtol=0.0, atol=None) -> Config:
    """A solver configuration.  rk=FR_BS32 selects adaptive steps: dt is the
    first proposed step, t_end / dt_max (<= 0: none) bound them, rtol and atol
    (a scalar or one value per conserved variable) set the error norm."""
    c = Config()
    c.gamma, c.prandtl, c.mu = gamma, prandtl, mu
    c.rho_inf, c.p_inf = rho_inf, p_inf
    v = [0.0, 0.0, 0.0] if v_inf is None else list(v_inf) + [0.0] * (3 - len(v_inf))
    for i in range(3):
        c.v_inf[i] = v[i]
    c.inflow_delta, c.inflow_ywall = inflow_delta, inflow_ywall
    c.br2_eta, c.dt = br2_eta, dt
    c.viscous, c.rk, c.precision, c.flux = int(bool(viscous)), rk, precision, flux
    c.viscous_scheme, c.ldg_beta, c.ldg_tau = viscous_scheme, ldg_beta, ldg_tau
    c.check_every = int(check_every)
    c.flux_reference = int(flux_reference)
    c.t_end, c.dt_max, c.rtol = float(t_end), float(dt_max), float(rtol)
    at = [0.0] * 5 if atol is None else (list(np.broadcast_to(np.asarray(atol, dtype=np.float64), (dim + 2,)))
                                         + [0.0] * (3 - dim))
    for i in range(5):
        c.atol[i] = at[i]
    return c


_lib = None


def lib():
    """Load libfr.so once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libfr.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(_LIB_PATH)
    P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
    dp = C.POINTER(C.c_double)
    L.fr_mesh_create.argtypes = [C.POINTER(P), I, I, I64, dp, I64, C.POINTER(C.c_int64), I, dp,
                                 C.POINTER(C.c_int32), I, dp]
    L.fr_mesh_create_varp.argtypes = [C.POINTER(P), I, C.POINTER(C.c_int32), I64, dp, I64,
                                      C.POINTER(C.c_int64), I, dp, C.POINTER(C.c_int32), I, dp]
    L.fr_mesh_degrees.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    L.fr_mesh_destroy.argtypes = [P]
    L.fr_mesh_destroy.restype = None
    L.fr_mesh_info.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(I), C.POINTER(I)]
    L.fr_mesh_sol_coords.argtypes = [P, dp]
    L.fr_workspace_bytes.argtypes = [C.POINTER(P), I, C.POINTER(Config)]
    L.fr_workspace_bytes.restype = C.c_size_t
    L.fr_solver_create.argtypes = [C.POINTER(P), C.POINTER(P), I, C.POINTER(Config), P, C.c_size_t, P]
    L.fr_solver_destroy.argtypes = [P]
    L.fr_solver_destroy.restype = None
    L.fr_set_state.argtypes = [P, I, dp]
    L.fr_get_state.argtypes = [P, I, dp]
    L.fr_set_states.argtypes = [P, dp]
    L.fr_accumulators_size.argtypes = [P]
    L.fr_accumulators_size.restype = C.c_int64
    L.fr_get_accumulators.argtypes = [P, dp]
    L.fr_set_accumulators.argtypes = [P, dp, I64]
    L.fr_get_states.argtypes = [P, dp]
    L.fr_residual.argtypes = [P, I, dp]
    L.fr_rk_step.argtypes = [P, I]
    L.fr_probe_add.argtypes = [P, I, dp, C.POINTER(I)]
    L.fr_probe_pressure.argtypes = [P, I, dp]
    L.fr_probe_reset.argtypes = [P]
    L.fr_probe_history.argtypes = [P, I, dp, I, C.POINTER(I)]
    L.fr_oaspl.argtypes = [P, C.POINTER(I), I, D, D, I, dp]
    L.fr_probe_stats.argtypes = [P, I, dp]
    L.fr_forces.argtypes = [P, I, dp]
    L.fr_conservation.argtypes = [P, I, dp]
    L.fr_integral.argtypes = [P, I, dp, C.POINTER(C.c_int64)]
    L.fr_integral_static.argtypes = [P, I, dp, C.POINTER(C.c_int64)]
    L.fr_instance_status.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(I)]
    L.fr_step_control.argtypes = [P, I, dp]
    L.fr_set_end_time.argtypes = [P, D]
    L.fr_force_coefficients.argtypes = [P, I, D, dp, dp]
    L.fr_tune.argtypes = [P, C.c_char_p, I, C.c_char_p, C.c_size_t]
    L.fr_schedule.argtypes = [P, C.c_char_p, C.c_size_t, C.c_char_p, C.c_size_t]
    L.fr_tune_lookup.argtypes = [C.c_char_p, C.c_char_p, C.c_char_p, C.c_size_t]
    L.fr_alu_peak.argtypes = [I, dp]
    L.fr_last_launch_count.argtypes = [P]
    L.fr_last_launch_count.restype = C.c_int64
    L.fr_profile_steps.argtypes = [P, I, dp, C.POINTER(C.c_int64)]
    L.fr_last_error.argtypes = []
    L.fr_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("fr_mesh_destroy", "fr_solver_destroy", "fr_workspace_bytes",
                        "fr_last_launch_count", "fr_last_error", "fr_accumulators_size"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def alu_peak(precision):
    """fr_alu_peak: measured FMA-pipe peak of the current GPU in flop/s."""
    out = C.c_double()
    _check(lib().fr_alu_peak(precision, C.byref(out)), "fr_alu_peak")
    return out.value


def tune_lookup(cache_path, key):
    """fr_tune_lookup (host only): the cached schedule under key, or None."""
    buf = C.create_string_buffer(256)
    st = lib().fr_tune_lookup(os.fsencode(cache_path), key.encode(), buf, 256)
    return buf.value.decode() if st == FR_OK else None


def _check(st, where):
    if st != FR_OK:
        raise FRError(st, where, lib().fr_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Mesh:
    """fr_mesh_create over a ``synth.meshes.Mesh``-like object (fields dim,
    xyz, elem_vert, face_tag, periodic_shift, geo_order, geo_nodes); ``p`` is
    one degree or one degree per element (fr_mesh_create_varp)."""

    def __init__(self, mesh, p):
        L = lib()
        self.dim = int(mesh.dim)
        varp = np.ndim(p) > 0
        self.p = None if varp else int(p)
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        ev = np.ascontiguousarray(mesh.elem_vert, dtype=np.int64)
        tags = np.ascontiguousarray(mesh.face_tag, dtype=np.int32)
        sh = np.ascontiguousarray(mesh.periodic_shift, dtype=np.float64).reshape(-1, self.dim)
        gn = None if getattr(mesh, "geo_nodes", None) is None else np.ascontiguousarray(mesh.geo_nodes, dtype=np.float64)
        q = int(getattr(mesh, "geo_order", 1))
        # the C call reads these arrays by the sizes it is given: check their shapes here
        if self.dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        if xyz.ndim != 2 or xyz.shape[1] != self.dim:
            raise ValueError(f"xyz must have shape (n_vert, {self.dim})")
        if ev.ndim != 2 or ev.shape[1] != 2 ** self.dim:
            raise ValueError(f"elem_vert must have shape (n_elem, {2 ** self.dim})")
        if tags.shape != (ev.shape[0], 2 * self.dim):
            raise ValueError(f"face_tag must have shape (n_elem, {2 * self.dim})")
        if gn is not None and (q < 1 or gn.size != ev.shape[0] * (q + 1) ** self.dim * self.dim):
            raise ValueError(f"geo_nodes must hold n_elem x (geo_order + 1)^{self.dim} x {self.dim} values")
        h = C.c_void_p()
        geo = (q, None if gn is None else _dptr(gn),
               tags.ctypes.data_as(C.POINTER(C.c_int32)), sh.shape[0], _dptr(sh) if sh.size else None)
        if varp:
            ep = np.ascontiguousarray(p, dtype=np.int32)
            if ep.shape != (ev.shape[0],):
                raise ValueError("one degree per element")
            st = L.fr_mesh_create_varp(C.byref(h), self.dim, ep.ctypes.data_as(C.POINTER(C.c_int32)),
                                       xyz.shape[0], _dptr(xyz), ev.shape[0],
                                       ev.ctypes.data_as(C.POINTER(C.c_int64)), *geo)
            _check(st, "fr_mesh_create_varp")
        else:
            st = L.fr_mesh_create(C.byref(h), self.dim, self.p, xyz.shape[0], _dptr(xyz), ev.shape[0],
                                  ev.ctypes.data_as(C.POINTER(C.c_int64)), *geo)
            _check(st, "fr_mesh_create")
        self.handle = h
        ne, nsp, nfp = C.c_int64(), C.c_int(), C.c_int()
        _check(L.fr_mesh_info(h, C.byref(ne), C.byref(nsp), C.byref(nfp)), "fr_mesh_info")
        self.n_elem, self.nsp, self.nfp = ne.value, nsp.value, nfp.value
        self.elem_p = np.empty(self.n_elem, dtype=np.int32)
        tot = C.c_int64()
        _check(L.fr_mesh_degrees(h, self.elem_p.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(tot)),
               "fr_mesh_degrees")
        self.n_sp = tot.value

    @property
    def state_shape(self):
        """Host state shape of one instance: (n_elem, nsp) for one degree,
        (n_sp,) element after element when the degree varies."""
        return (self.n_elem, self.nsp) if self.nsp else (self.n_sp,)

    def sol_coords(self):
        out = np.empty(self.state_shape + (self.dim,))
        _check(lib().fr_mesh_sol_coords(self.handle, _dptr(out)), "fr_mesh_sol_coords")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().fr_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """fr_solver_create over a batch of Mesh objects; device workspace and
    stream come from PyTorch."""

    def __init__(self, meshes, cfg: Config, device="cuda", stream=None):
        import torch
        L = lib()
        self.meshes = list(meshes)
        self.cfg = cfg
        self.dim = self.meshes[0].dim
        self.V = self.dim + 2
        arr = (C.c_void_p * len(self.meshes))(*[m.handle for m in self.meshes])
        self._arr = arr
        nbytes = L.fr_workspace_bytes(arr, len(self.meshes), C.byref(cfg))
        if nbytes == 0:
            raise FRError(1, "fr_workspace_bytes", L.fr_last_error().decode())
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        h = C.c_void_p()
        torch.cuda.synchronize(device)
        st = L.fr_solver_create(C.byref(h), arr, len(self.meshes), C.byref(cfg), C.c_void_p(aligned),
                                nbytes, C.c_void_p(self.stream.cuda_stream))
        _check(st, "fr_solver_create")
        self.handle = h
        self.ws_bytes = nbytes

    def n_elem(self, inst):
        return self.meshes[inst].n_elem

    def set_state(self, inst, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        m = self.meshes[inst]
        if u.shape != m.state_shape + (self.V,):
            raise ValueError("state shape")
        _check(lib().fr_set_state(self.handle, inst, _dptr(u)), "fr_set_state")

    def _out(self, inst, out):
        shape = self.meshes[inst].state_shape + (self.V,)
        if out is None:
            return np.empty(shape)
        if (not isinstance(out, np.ndarray) or out.dtype != np.float64 or out.shape != shape
                or not out.flags.c_contiguous or not out.flags.writeable):
            raise ValueError(f"out must be a writeable C-contiguous float64 array of shape {shape}")
        return out

    def get_state(self, inst, out=None):
        """FP64 state of one instance; ``out`` (optional) is written in place,
        e.g. a pinned host buffer so that the copy runs at full link speed."""
        out = self._out(inst, out)
        _check(lib().fr_get_state(self.handle, inst, _dptr(out)), "fr_get_state")
        return out

    def state_sizes(self):
        """Number of FP64 values of each instance's state."""
        return [int(np.prod(m.state_shape)) * self.V for m in self.meshes]

    def set_states(self, u):
        """All instances at once from one flat FP64 array (instance after
        instance), one synchronisation (fr_set_states)."""
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        if u.size != sum(self.state_sizes()):
            raise ValueError("state size")
        _check(lib().fr_set_states(self.handle, _dptr(u)), "fr_set_states")

    def get_states(self, out=None):
        """All instances' states into one flat FP64 array (``out`` written in
        place when given, e.g. pinned host memory); returns it."""
        n = sum(self.state_sizes())
        if out is None:
            out = np.empty(n)
        elif (not isinstance(out, np.ndarray) or out.dtype != np.float64 or out.size != n
              or not out.flags.c_contiguous or not out.flags.writeable):
            raise ValueError(f"out must be a writeable C-contiguous float64 array of {n} values")
        _check(lib().fr_get_states(self.handle, _dptr(out)), "fr_get_states")
        return out

    def get_accumulators(self):
        """Checkpoint of the observers and wall-force sums (fr_get_accumulators)."""
        out = np.empty(int(lib().fr_accumulators_size(self.handle)))
        _check(lib().fr_get_accumulators(self.handle, _dptr(out)), "fr_get_accumulators")
        return out

    def set_accumulators(self, acc):
        acc = np.ascontiguousarray(acc, dtype=np.float64)
        if acc.size != int(lib().fr_accumulators_size(self.handle)):
            raise ValueError("accumulator checkpoint size")
        _check(lib().fr_set_accumulators(self.handle, _dptr(acc), acc.size), "fr_set_accumulators")

    def residual(self, inst, out=None):
        out = self._out(inst, out)
        _check(lib().fr_residual(self.handle, inst, _dptr(out)), "fr_residual")
        return out

    def rk_step(self, n):
        _check(lib().fr_rk_step(self.handle, int(n)), "fr_rk_step")

    def last_launch_count(self):
        return int(lib().fr_last_launch_count(self.handle))

    def probe_add(self, inst, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        if x.size != self.dim:
            raise ValueError(f"probe point needs {self.dim} coordinates")
        pid = C.c_int()
        _check(lib().fr_probe_add(self.handle, inst, _dptr(x), C.byref(pid)), "fr_probe_add")
        return pid.value

    def probe_pressure(self, pid):
        v = C.c_double()
        _check(lib().fr_probe_pressure(self.handle, pid, C.byref(v)), "fr_probe_pressure")
        return v.value

    def probe_history(self, pid, max_n=4096):
        out = np.empty(max_n)
        n = C.c_int()
        _check(lib().fr_probe_history(self.handle, pid, _dptr(out), max_n, C.byref(n)), "fr_probe_history")
        return out[:n.value].copy()

    def probe_stats(self, pid):
        out = np.empty(4)
        _check(lib().fr_probe_stats(self.handle, pid, _dptr(out)), "fr_probe_stats")
        return out

    def probe_reset(self):
        _check(lib().fr_probe_reset(self.handle), "fr_probe_reset")

    def oaspl(self, pids, p_ref=2e-5, p_scale=1.0, mean_mode=0):
        ids = (C.c_int * len(pids))(*pids)
        v = C.c_double()
        _check(lib().fr_oaspl(self.handle, ids, len(pids), p_ref, p_scale, mean_mode, C.byref(v)),
               "fr_oaspl")
        return v.value

    def forces(self, inst):
        out = np.zeros(3)
        _check(lib().fr_forces(self.handle, inst, _dptr(out)), "fr_forces")
        return out[:self.dim]

    def force_coefficients(self, inst, a_ref):
        """(mean C_L, mean C_D) of fr_force_coefficients."""
        cl, cd = C.c_double(), C.c_double()
        _check(lib().fr_force_coefficients(self.handle, inst, a_ref, C.byref(cl), C.byref(cd)),
               "fr_force_coefficients")
        return cl.value, cd.value

    def conservation(self, inst):
        out = np.zeros(self.V)
        _check(lib().fr_conservation(self.handle, inst, _dptr(out)), "fr_conservation")
        return out

    def integral(self, inst):
        out = np.zeros(self.V)
        bad = C.c_int64()
        st = lib().fr_integral(self.handle, inst, _dptr(out), C.byref(bad))
        if st not in (0, 5):
            _check(st, "fr_integral")
        return out, bad.value

    def profile_steps(self, n):
        """Mean ms per launch and launch counts per kernel kind:
        (flux, gradient, probe, force, other)."""
        ms = np.zeros(5)
        cnt = np.zeros(5, dtype=np.int64)
        _check(lib().fr_profile_steps(self.handle, int(n), _dptr(ms),
                                      cnt.ctypes.data_as(C.POINTER(C.c_int64))), "fr_profile_steps")
        return ms, cnt

    def integral_static(self, inst):
        """fr_integral without workspace scratch (reduction scratch in a
        fixed device array inside the library); raises FRError for instances
        above its size limit."""
        out = np.zeros(self.V)
        bad = C.c_int64()
        st = lib().fr_integral_static(self.handle, inst, _dptr(out), C.byref(bad))
        if st not in (0, 5):
            _check(st, "fr_integral_static")
        return out, bad.value

    def tune(self, cache_path=None, mode=0):
        """fr_tune: measure (or look up) the stage schedule; returns the
        choice string.  Call before set_state (it starts from the free
        stream)."""
        buf = C.create_string_buffer(512)
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(lib().fr_tune(self.handle, path, mode, buf, 512), "fr_tune")
        return buf.value.decode()

    def schedule(self):
        """(schedule string, cache key) of fr_schedule."""
        a, b = C.create_string_buffer(256), C.create_string_buffer(256)
        _check(lib().fr_schedule(self.handle, a, 256, b, 256), "fr_schedule")
        return a.value.decode(), b.value.decode()

    def instance_status(self):
        """(flags, first_bad) of fr_instance_status: one flag per instance,
        set where a scan found NaN/Inf (needs check_every > 0 in the config);
        first_bad = -1 when none."""
        flags = np.zeros(len(self.meshes), dtype=np.int32)
        first = C.c_int()
        st = lib().fr_instance_status(self.handle, flags.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(first))
        if st not in (0, 5):
            _check(st, "fr_instance_status")
        return flags, first.value

    def step_control(self, inst):
        """Step-control record of one instance (adaptive steps, FR_BS32)."""
        out = np.zeros(8)
        _check(lib().fr_step_control(self.handle, inst, out.ctypes.data_as(C.POINTER(C.c_double))),
               "fr_step_control")
        keys = ("t", "h", "h_next", "err", "rejected_in_step", "accepted", "rejected", "samples")
        return dict(zip(keys, out.tolist()))

    def set_end_time(self, t_end):
        """Adaptive steps: move every instance's end time (fr_set_end_time)."""
        _check(lib().fr_set_end_time(self.handle, float(t_end)), "fr_set_end_time")

    def advance_to(self, t_end, chunk=50, max_attempts=100000):
        """Adaptive steps: attempts until every instance has reached t_end
        (checked every `chunk` attempts), at most max_attempts.  Returns one
        flag per instance: True where t_end was reached (False means the
        step size collapsed, e.g. on a diverging flow)."""
        self.set_end_time(t_end)
        n = len(self.meshes)
        done = 0
        reached = np.zeros(n, dtype=bool)
        while done < max_attempts:
            k = min(chunk, max_attempts - done)
            self.rk_step(k)
            done += k
            reached = np.array([self.step_control(i)["t"] >= t_end for i in range(n)])
            if reached.all():
                break
        return reached

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "handle", None):
            lib().fr_solver_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
