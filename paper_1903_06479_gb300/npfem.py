"""ctypes binding of libnpfem.so (include/npfem.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; there is no CPU path.
Device arrays may be passed as torch tensors (their data_ptr is used) or as raw
integer addresses.  Errors raise NpfemError with the library's message."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
CELL_STATUS = {0: "OK", 1: "MAXITER", 2: "LINESEARCH_FAIL", 3: "NONFINITE"}
MATERIAL_ORDER = ("B", "C", "D", "k_bend", "k_vol", "k_mat_hess", "density", "alpha_D", "beta_D", "kappa")


class NpfemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"npfem error {code}: {msg}")
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32), ("tris", C.c_void_p), ("rest_xyz", C.c_void_p)]


class Material(C.Structure):
    _fields_ = [(k, C.c_double) for k in MATERIAL_ORDER]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("lbfgs_m", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("c1", C.c_double), ("c2", C.c_double), ("max_halvings", C.c_int32), ("fixed_alpha", C.c_int32),
                ("equal_mass", C.c_int32), ("armijo_noise", C.c_double), ("refine", C.c_int32),
                ("fill_idle_sms", C.c_int32), ("warm_history", C.c_int32)]


class Lattice(C.Structure):
    """npfem_lattice: node (i, j, k) at origin + dx (i, j, k)."""
    _fields_ = [("origin", C.c_double * 3), ("dx", C.c_double), ("nx", C.c_int32), ("ny", C.c_int32),
                ("nz", C.c_int32), ("reserved", C.c_int32)]


def lattice(origin, dx, shape_xyz) -> Lattice:
    return Lattice((C.c_double * 3)(*[float(o) for o in origin]), float(dx), *[int(s) for s in shape_xyz], 0)


class CellStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("evaluations", C.c_int32), ("status", C.c_int32),
                ("residual", C.c_float), ("objective", C.c_double), ("volume", C.c_double)]


CELL_STATS_DTYPE = np.dtype([("iterations", "<i4"), ("evaluations", "<i4"), ("status", "<i4"),
                             ("residual", "<f4"), ("objective", "<f8"), ("volume", "<f8")])

_lib = None
EXPORTS = ("npfem_default_opts", "npfem_create", "npfem_destroy", "npfem_step", "npfem_step_host", "npfem_eval",
           "npfem_get_inverse", "npfem_get_rest_info", "npfem_last_error", "npfem_step_static",
           "npfem_check_device", "npfem_mlp_nparam", "npfem_ws_features", "npfem_mlp_loss_grad", "npfem_mlp_adam",
           "npfem_mlp_predict", "npfem_set_warmstart", "npfem_ws_guess", "npfem_launch_count",
           "npfem_kernel_timing", "npfem_kernel_times", "npfem_graph_create", "npfem_graph_launch",
           "npfem_graph_destroy", "npfem_kernel_time_last", "npfem_autotune", "npfem_get_tuning",
           "npfem_flag_wait_timeout", "npfem_ibm_forces", "npfem_ibm_interpolate", "npfem_ibm_forcing",
           "npfem_collision_detect", "npfem_set_collisions", "npfem_set_warmstart_temporal",
           "npfem_ws_features_temporal", "npfem_ws_guess_temporal")


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads libnpfem.so (building it first if a source is newer); raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i32 = C.c_void_p, C.c_int
        L.npfem_graph_create.argtypes = [vp, i32, vp, vp, vp, vp, C.c_double, i32, vp, C.POINTER(vp)]
        L.npfem_graph_launch.argtypes = [vp, vp]
        L.npfem_graph_destroy.argtypes = [vp]
        L.npfem_kernel_time_last.argtypes = [vp, vp]
        L.npfem_autotune.argtypes = [vp, i32, vp, vp, vp, vp, C.c_double, i32, vp]
        L.npfem_get_tuning.argtypes = [vp, vp, vp, vp]
        L.npfem_kernel_timing.argtypes = [vp, i32]
        L.npfem_kernel_times.argtypes = [vp, vp, i32, vp]
        L.npfem_launch_count.argtypes = []
        L.npfem_launch_count.restype = C.c_ulonglong
        L.npfem_default_opts.argtypes = [C.POINTER(Opts)]
        L.npfem_default_opts.restype = None
        L.npfem_create.argtypes = [C.POINTER(Mesh), C.POINTER(Material), C.POINTER(Opts), C.c_double, i32, C.POINTER(vp)]
        L.npfem_destroy.argtypes = [vp]
        L.npfem_step.argtypes = [C.POINTER(vp), i32, C.POINTER(C.c_int32), vp, vp, vp, C.c_double, vp, vp]
        L.npfem_step_static.argtypes = [C.POINTER(vp), i32, C.POINTER(C.c_int32), vp, vp, vp, C.c_double, vp, vp]
        L.npfem_step_host.argtypes = [vp, i32, vp, vp, vp, C.c_double, vp, vp]
        L.npfem_eval.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.npfem_get_inverse.argtypes = [vp, vp]
        L.npfem_get_rest_info.argtypes = [vp, vp, vp]
        L.npfem_check_device.argtypes = [vp]
        L.npfem_flag_wait_timeout.argtypes = [vp]
        L.npfem_set_warmstart_temporal.argtypes = [vp, vp]
        L.npfem_ws_features_temporal.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.npfem_ws_guess_temporal.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.npfem_collision_detect.argtypes = [vp, i32, vp, vp, C.c_double, vp, vp, vp]
        L.npfem_set_collisions.argtypes = [vp, vp, C.c_double]
        L.npfem_ibm_forces.argtypes = [vp, i32, vp, vp, C.POINTER(Lattice), vp, C.c_double, i32, vp, vp]
        L.npfem_ibm_interpolate.argtypes = [vp, i32, vp, vp, C.POINTER(Lattice), vp, vp, vp]
        L.npfem_ibm_forcing.argtypes = [vp, i32, vp, vp, vp, C.POINTER(Lattice), vp, C.c_double, i32, vp, vp, vp]
        L.npfem_mlp_nparam.argtypes = []
        L.npfem_ws_features.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
        L.npfem_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
        L.npfem_mlp_adam.argtypes = [vp, vp, vp, vp, i32, C.c_float, C.c_float, C.c_float, C.c_float, vp]
        L.npfem_mlp_predict.argtypes = [vp, vp, i32, vp, vp, vp]
        L.npfem_set_warmstart.argtypes = [vp, vp, i32]
        L.npfem_ws_guess.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.npfem_last_error.restype = C.c_char_p
        L.npfem_last_error.argtypes = []
        for name in EXPORTS:
            if name not in ("npfem_default_opts", "npfem_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise NpfemError(rc, lib().npfem_last_error().decode())


def _addr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().npfem_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PREC[v]
        setattr(o, k, v)
    return o


def material(**kw) -> Material:
    from .workloads import DEFAULT_MATERIAL
    d = dict(DEFAULT_MATERIAL)
    d.update(kw)
    return Material(*[float(d[k]) for k in MATERIAL_ORDER])


class Handle:
    """One mesh topology on one device (npfem_create / npfem_destroy)."""

    def __init__(self, rest: np.ndarray, tris: np.ndarray, mat: Material | None = None, opts: Opts | None = None,
                 dt: float = 0.1, device: int = 0):
        self._rest = np.ascontiguousarray(rest, dtype=np.float64)
        self._tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.n = self._rest.shape[0]
        self.nt = self._tris.shape[0]
        self.opts = opts or default_opts()
        self.material = mat or material()
        self.dt = float(dt)
        self.device = device
        self.precision = int(self.opts.precision)
        m = Mesh(self.n, self.nt, self._tris.ctypes.data, self._rest.ctypes.data)
        h = C.c_void_p()
        _check(lib().npfem_create(C.byref(m), C.byref(self.material), C.byref(self.opts), self.dt, device, C.byref(h)))
        self._h = h

    @property
    def ptr(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().npfem_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_warmstart(self, params: np.ndarray | None, mode: int = 1):
        """Installs a trained warm-start network (5016 FP32 parameters) or removes it."""
        if params is None:
            _check(lib().npfem_set_warmstart(self._h, None, 0))
        else:
            p = np.ascontiguousarray(params, dtype=np.float32)
            assert p.size == mlp_nparam()
            _check(lib().npfem_set_warmstart(self._h, p.ctypes.data, int(mode)))

    def ws_features(self, n_cells, x, v, f, feat, x_next=None, target=None, stream=None):
        _check(lib().npfem_ws_features(self._h, n_cells, _addr(x), _addr(v), _addr(f), _addr(x_next), _addr(feat),
                                       _addr(target), _addr(stream)))

    def set_warmstart_temporal(self, params: np.ndarray | None):
        """Installs (5016 FP32 parameters) or removes the temporal network."""
        if params is None:
            _check(lib().npfem_set_warmstart_temporal(self._h, None))
        else:
            p = np.ascontiguousarray(params, dtype=np.float32)
            assert p.size == mlp_nparam()
            _check(lib().npfem_set_warmstart_temporal(self._h, p.ctypes.data))

    def ws_features_temporal(self, n_cells, x, v, f, f_prev, c1, c2, feat, x_next=None, target=None, c_out=None,
                             stream=None):
        _check(lib().npfem_ws_features_temporal(self._h, n_cells, _addr(x), _addr(v), _addr(f), _addr(f_prev),
                                                _addr(c1), _addr(c2), _addr(x_next), _addr(feat), _addr(target),
                                                _addr(c_out), _addr(stream)))

    def ws_guess_temporal(self, n_cells, x, v, f, f_prev, c1, c2, u_out, stream=None):
        _check(lib().npfem_ws_guess_temporal(self._h, n_cells, _addr(x), _addr(v), _addr(f), _addr(f_prev), _addr(c1),
                                             _addr(c2), _addr(u_out), _addr(stream)))

    def ws_guess(self, n_cells, x, v, f, x1, stream=None):
        _check(lib().npfem_ws_guess(self._h, n_cells, _addr(x), _addr(v), _addr(f), _addr(x1), _addr(stream)))

    def check_device(self):
        """Raises NpfemError(-5) if a bounded device wait of a previous step gave up."""
        _check(lib().npfem_check_device(self._h))

    def set_collisions(self, planes, w_col: float):
        """npfem_set_collisions: collision planes (device) for the steps through this handle."""
        _check(lib().npfem_set_collisions(self._h, _addr(planes), float(w_col) if planes is not None else 0.0))

    def flag_wait_timeout(self):
        """Sets the device-wait flag as a timed-out wait would (tests the reporting path)."""
        _check(lib().npfem_flag_wait_timeout(self._h))

    def inverse(self) -> np.ndarray:
        out = np.zeros((self.n, self.n))
        _check(lib().npfem_get_inverse(self._h, out.ctypes.data))
        return out

    def rest_info(self):
        m = np.zeros(self.n)
        s = np.zeros(4)
        _check(lib().npfem_get_rest_info(self._h, m.ctypes.data, s.ctypes.data))
        return m, dict(V0=s[0], A0=s[1], lbar=s[2], mtotal=s[3])

    def kernel_timing(self, capacity: int):
        """Record the solver-kernel time of the next `capacity` steps (0: stop)."""
        _check(lib().npfem_kernel_timing(self._h, int(capacity)))

    def tuning(self) -> dict:
        """The launch shape this handle uses (npfem_get_tuning)."""
        t, th, fi = C.c_int(0), C.c_int(0), C.c_int(0)
        _check(lib().npfem_get_tuning(self._h, C.addressof(t), C.addressof(th), C.addressof(fi)))
        return {"tensor_core": bool(t.value), "simt_threads": th.value, "fill_idle_sms": bool(fi.value)}

    def kernel_time_last(self) -> float:
        """Duration (ms) of the first recorded solver launch pair (latest graph replay)."""
        ms = C.c_float(0.0)
        _check(lib().npfem_kernel_time_last(self._h, C.addressof(ms)))
        return float(ms.value)

    def kernel_times(self, max_n: int = 4096) -> np.ndarray:
        """Durations (ms) of the recorded solver launches; restarts the recording."""
        out = np.zeros(max_n, dtype=np.float32)
        n = C.c_int(0)
        _check(lib().npfem_kernel_times(self._h, out.ctypes.data, int(max_n), C.addressof(n)))
        return out[:n.value].copy()

    def eval(self, n_cells: int, x, y, grad, parts, stream=None):
        _check(lib().npfem_eval(self._h, n_cells, _addr(x), _addr(y), _addr(grad), _addr(parts), _addr(stream)))

    def step_host(self, x: np.ndarray, v: np.ndarray, f: np.ndarray, stats: np.ndarray | None = None, stream=None):
        """One step of x, v (host SoA arrays, updated in place) with host forces f."""
        n_cells = x.shape[0]
        _check(lib().npfem_step_host(self._h, n_cells, x.ctypes.data, v.ctypes.data, f.ctypes.data, self.dt,
                                     _addr(stream), None if stats is None else stats.ctypes.data))


def step(handles, cells_per_group, x, v, f, dt: float, stream=None, stats=None):
    """npfem_step over one or more handles (device SoA state, updated in place)."""
    handles = list(handles)
    arr = (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    cells = (C.c_int32 * len(handles))(*[int(c) for c in cells_per_group])
    _check(lib().npfem_step(arr, len(handles), cells, _addr(x), _addr(v), _addr(f), float(dt), _addr(stream),
                            _addr(stats)))


def autotune(handles, cells_per_group, x, v, f, dt: float, trial_steps: int = 2):
    """npfem_autotune: picks each handle's launch shape by timing trial steps on copies
    of its cells; returns the chosen shapes."""
    handles = list(handles)
    arr = (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    cells = (C.c_int32 * len(handles))(*[int(c) for c in cells_per_group])
    ms = np.zeros(5 * len(handles), dtype=np.float32)
    _check(lib().npfem_autotune(arr, len(handles), cells, _addr(x), _addr(v), _addr(f), float(dt), int(trial_steps),
                                ms.ctypes.data))
    names = ("simt512", "simt640", "tc_fill512", "tc_only", "tc_fill640")
    out = []
    for g, h in enumerate(handles):
        t = h.tuning()
        t["trial_ms"] = {nm: float(ms[5 * g + q]) for q, nm in enumerate(names) if ms[5 * g + q] >= 0}
        out.append(t)
    return out


class StepGraph:
    """npfem_graph_*: `steps` consecutive npfem_step calls on fixed buffers captured as
    one CUDA graph; launch() replays them on a stream.  Keep the handles alive."""

    def __init__(self, handles, cells_per_group, x, v, f, dt: float, steps: int = 1, stats=None):
        handles = list(handles)
        self._handles = handles
        arr = (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])
        cells = (C.c_int32 * len(handles))(*[int(c) for c in cells_per_group])
        self._g = C.c_void_p()
        _check(lib().npfem_graph_create(arr, len(handles), cells, _addr(x), _addr(v), _addr(f), float(dt), int(steps),
                                        _addr(stats), C.byref(self._g)))
        self.steps = steps

    def launch(self, stream=None):
        _check(lib().npfem_graph_launch(self._g, _addr(stream)))

    def close(self):
        if self._g:
            lib().npfem_graph_destroy(self._g)
            self._g = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _groups(handles, cells_per_group):
    handles = list(handles)
    arr = (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    cells = (C.c_int32 * len(handles))(*[int(c) for c in cells_per_group])
    return arr, len(handles), cells


def ibm_forces(handles, cells_per_group, x, lat: Lattice, sigma, f_out, rho_fluid=1.0, mode=0, stream=None):
    """npfem_ibm_forces: Eq. Fext from a lattice stress field into f_out (device SoA)."""
    arr, ng, cells = _groups(handles, cells_per_group)
    _check(lib().npfem_ibm_forces(arr, ng, cells, _addr(x), C.byref(lat), _addr(sigma), float(rho_fluid), int(mode),
                                  _addr(f_out), _addr(stream)))


def ibm_interpolate(handles, cells_per_group, x, lat: Lattice, u_lattice, u_out, stream=None):
    arr, ng, cells = _groups(handles, cells_per_group)
    _check(lib().npfem_ibm_interpolate(arr, ng, cells, _addr(x), C.byref(lat), _addr(u_lattice), _addr(u_out),
                                       _addr(stream)))


def ibm_forcing(handles, cells_per_group, x, u_vertex, lat: Lattice, u_lattice, dt_fluid, cycles, f_vertex, f_lattice,
                stream=None):
    """npfem_ibm_forcing: multi-direct forcing; writes f_vertex (SoA) and f_lattice."""
    arr, ng, cells = _groups(handles, cells_per_group)
    _check(lib().npfem_ibm_forcing(arr, ng, cells, _addr(x), _addr(u_vertex), C.byref(lat), _addr(u_lattice),
                                   float(dt_fluid), int(cycles), _addr(f_vertex), _addr(f_lattice), _addr(stream)))


def collision_detect(handles, cells_per_group, x, cutoff: float, planes, stats, stream=None):
    """npfem_collision_detect: per-vertex planes of the nearest vertex of another cell."""
    arr, ng, cells = _groups(handles, cells_per_group)
    _check(lib().npfem_collision_detect(arr, ng, cells, _addr(x), float(cutoff), _addr(planes), _addr(stats),
                                        _addr(stream)))


def step_static(handles, cells_per_group, x, v, f, dt: float, stream=None, stats=None):
    """npfem_step_static: npfem_step without any device allocation (fixed library scratch)."""
    handles = list(handles)
    arr = (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    cells = (C.c_int32 * len(handles))(*[int(c) for c in cells_per_group])
    _check(lib().npfem_step_static(arr, len(handles), cells, _addr(x), _addr(v), _addr(f), float(dt), _addr(stream),
                                   _addr(stats)))


def launch_count() -> int:
    """Kernels the library has launched so far in this process."""
    return int(lib().npfem_launch_count())


def mlp_nparam() -> int:
    return lib().npfem_mlp_nparam()


def mlp_loss_grad(params, feat, target, idx, n, grad, loss, stream=None):
    """Mean loss and gradient of the warm-start network over n samples (device pointers)."""
    _check(lib().npfem_mlp_loss_grad(_addr(params), _addr(feat), _addr(target), _addr(idx), int(n), _addr(grad),
                                     _addr(loss), _addr(stream)))


def mlp_adam(params, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().npfem_mlp_adam(_addr(params), _addr(m), _addr(v), _addr(grad), int(step), float(lr), float(beta1),
                                float(beta2), float(eps), _addr(stream)))


def mlp_predict(params, feat, n, out, scratch, stream=None):
    _check(lib().npfem_mlp_predict(_addr(params), _addr(feat), int(n), _addr(out), _addr(scratch), _addr(stream)))
