"""ctypes wrapper of the FP64 CPU oracle (npfem_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product package.

Arrays are float64, AoS [n, 3] per cell (or [cells, n, 3] for batches).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "npfem_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libnpfem_oracle.so")

MATERIAL_ORDER = ("B", "C", "D", "k_bend", "k_vol", "k_mat_hess", "density", "alpha_D", "beta_D", "kappa")
STATUS = {0: "OK", 1: "MAXITER", 2: "LINESEARCH_FAIL", 3: "NONFINITE"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, SRC, "-lm", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


class Opts(C.Structure):
    _fields_ = [("lbfgs_m", C.c_int), ("max_iter", C.c_int), ("tol", C.c_double), ("c1", C.c_double),
                ("c2", C.c_double), ("max_halvings", C.c_int), ("fixed_alpha", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("evaluations", C.c_int), ("status", C.c_int), ("pad", C.c_int),
                ("residual", C.c_double), ("objective", C.c_double), ("volume", C.c_double), ("area", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        L.or_create.restype = P
        L.or_create.argtypes = [C.c_int, C.c_int, ip, dp, dp, C.c_double, C.c_int]
        L.or_destroy.argtypes = [P]
        L.or_rest_info.argtypes = [P, dp]
        for name in ("or_masses", "or_voronoi", "or_laplacian", "or_hessian", "or_apply_hinv"):
            getattr(L, name).argtypes = [P, dp]
        L.or_sl2_project.restype = C.c_double
        L.or_sl2_project.argtypes = [C.c_double, C.c_double]
        for name in ("or_skalak_f", "or_skalak_fp"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double, C.c_double, C.c_double]
        for name in ("or_energy_area", "or_energy_skalak"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [P, dp, P, P]
        L.or_energy_bend.restype = C.c_double
        L.or_energy_bend.argtypes = [P, dp, P]
        L.or_energy_vol.restype = C.c_double
        L.or_energy_vol.argtypes = [P, dp, P, P]
        L.or_volume.restype = C.c_double
        L.or_volume.argtypes = [P, dp]
        L.or_area.restype = C.c_double
        L.or_area.argtypes = [P, dp]
        L.or_volume_gradient.argtypes = [P, dp, dp]
        L.or_objective.restype = C.c_double
        L.or_objective.argtypes = [P, dp, dp, P, P, P]
        L.or_internal_energy.restype = C.c_double
        L.or_internal_energy.argtypes = [P, dp, P]
        L.or_first_guess.argtypes = [P, dp, dp, dp, dp]
        L.or_residual.restype = C.c_double
        L.or_residual.argtypes = [P, dp]
        L.or_solve.restype = C.c_int
        L.or_solve.argtypes = [P, dp, dp, C.POINTER(Opts), C.POINTER(Stats)]
        L.or_solve_carry.restype = C.c_int
        L.or_solve_carry.argtypes = [P, dp, dp, C.POINTER(Opts), C.POINTER(Stats), dp, dp, C.POINTER(C.c_int)]
        L.or_post_step.argtypes = [P, dp, dp, C.c_double]
        L.or_step.restype = C.c_int
        L.or_step.argtypes = [P, dp, dp, dp, C.POINTER(Opts), C.POINTER(Stats)]
        L.or_mlp_nparam.restype = C.c_int
        L.or_bf16.restype = C.c_double
        L.or_bf16.argtypes = [C.c_double]
        L.or_mlp_predict.argtypes = [dp, dp, C.c_int, dp, C.c_int]
        L.or_mlp_loss_grad.restype = C.c_double
        L.or_mlp_loss_grad.argtypes = [dp, dp, dp, C.c_int, dp, C.c_int]
        L.or_best_rotation.argtypes = [P, dp, dp, dp, dp]
        L.or_ws_features.argtypes = [P, dp, dp, dp, dp]
        L.or_ws_guess.argtypes = [P, dp, dp, dp, dp, dp, C.c_int]
        L.or_objective_col.restype = C.c_double
        L.or_objective_col.argtypes = [P, dp, dp, P, P, P, P, C.c_double]
        L.or_energy_collision.restype = C.c_double
        L.or_energy_collision.argtypes = [P, dp, P, C.c_double, P]
        L.or_step_col.restype = C.c_int
        L.or_step_col.argtypes = [P, dp, dp, dp, C.POINTER(Opts), C.POINTER(Stats), P, C.c_double]
        L.or_step_batch_col.restype = C.c_int
        L.or_step_batch_col.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, C.POINTER(Opts), C.POINTER(Stats), C.c_int,
                                        P, C.c_double]
        L.or_ws_features_temporal.argtypes = [P, dp, dp, dp, dp, dp, dp, dp]
        L.or_ws_guess_temporal.argtypes = [P, dp, dp, dp, dp, dp, dp, dp, dp, C.c_int]
        L.or_step_batch.restype = C.c_int
        L.or_step_batch.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, C.POINTER(Opts), C.POINTER(Stats), C.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def make_opts(lbfgs_m=5, max_iter=50, tol=1e-6, c1=1e-4, c2=0.9, max_halvings=30, fixed_alpha=0) -> Opts:
    return Opts(lbfgs_m, max_iter, tol, c1, c2, max_halvings, fixed_alpha)


def sl2_project(s1: float, s2: float) -> float:
    return lib().or_sl2_project(float(s1), float(s2))


def skalak_f(l, B, D):
    return lib().or_skalak_f(float(l), float(B), float(D))


def skalak_fp(l, B, D):
    return lib().or_skalak_fp(float(l), float(B), float(D))


def mlp_nparam() -> int:
    return lib().or_mlp_nparam()


def bf16(x: float) -> float:
    return lib().or_bf16(float(x))


def mlp_predict(P, feat, bf16_operands=True):
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    out = np.zeros((feat.shape[0], 3))
    lib().or_mlp_predict(np.ascontiguousarray(P, dtype=np.float64), feat, feat.shape[0], out, int(bf16_operands))
    return out


def mlp_loss_grad(P, feat, target, bf16_operands=True):
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    g = np.zeros(mlp_nparam())
    loss = lib().or_mlp_loss_grad(np.ascontiguousarray(P, dtype=np.float64), feat,
                                  np.ascontiguousarray(target, dtype=np.float64), feat.shape[0], g, int(bf16_operands))
    return loss, g


class Model:
    """One mesh topology with its rest shape, material and time step."""

    def __init__(self, rest: np.ndarray, tris: np.ndarray, material: np.ndarray, dt: float, equal_mass: bool = False):
        L = lib()
        self.rest = np.ascontiguousarray(rest, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.material = np.ascontiguousarray(material, dtype=np.float64)
        self.dt = float(dt)
        self.n = self.rest.shape[0]
        self._h = L.or_create(self.n, self.tris.shape[0], self.tris, self.rest, self.material, self.dt, int(equal_mass))
        if not self._h:
            raise ValueError("oracle rejected the mesh (not a closed oriented manifold, or H~ not SPD)")
        info = np.zeros(4)
        L.or_rest_info(self._h, info)
        self.V0, self.A0, self.lbar, self.mtotal = info

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_destroy(self._h)
            self._h = None

    # --- queries -----------------------------------------------------------------
    def masses(self):
        o = np.zeros(self.n); lib().or_masses(self._h, o); return o

    def voronoi(self):
        o = np.zeros(self.n); lib().or_voronoi(self._h, o); return o

    def laplacian(self):
        o = np.zeros((self.n, self.n)); lib().or_laplacian(self._h, o); return o

    def hessian(self):
        o = np.zeros((self.n, self.n)); lib().or_hessian(self._h, o); return o

    def apply_hinv(self, b):
        b = np.array(b, dtype=np.float64, order="C"); lib().or_apply_hinv(self._h, b); return b

    # --- energies ------------------------------------------------------------------
    def _energy(self, fn, x, with_grad=True):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.zeros_like(x) if with_grad else None
        bad = C.c_int(0)
        e = fn(self._h, x, _ptr(g), C.byref(bad))
        return e, g

    def energy_area(self, x):
        return self._energy(lib().or_energy_area, x)

    def energy_skalak(self, x):
        return self._energy(lib().or_energy_skalak, x)

    def energy_bend(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.zeros_like(x)
        return lib().or_energy_bend(self._h, x, _ptr(g)), g

    def energy_vol(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.zeros_like(x)
        V = C.c_double(0)
        e = lib().or_energy_vol(self._h, x, _ptr(g), C.byref(V))
        return e, g

    def volume(self, x):
        return lib().or_volume(self._h, np.ascontiguousarray(x, dtype=np.float64))

    def area(self, x):
        return lib().or_area(self._h, np.ascontiguousarray(x, dtype=np.float64))

    def volume_gradient(self, x):
        o = np.zeros((self.n, 3)); lib().or_volume_gradient(self._h, np.ascontiguousarray(x, dtype=np.float64), o); return o

    def objective(self, x, y):
        """g(x) and grad g(x); parts = (inertia, area, skalak, bend, volume energy, V)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        g = np.zeros_like(x)
        parts = np.zeros(6)
        bad = C.c_int(0)
        e = lib().or_objective(self._h, x, y, _ptr(g), _ptr(parts), C.byref(bad))
        return e, g, parts

    def objective_col(self, x, y, col, wcol):
        """g(x) and grad g(x) with the collision term of planes col [n, 4]."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        col = np.ascontiguousarray(col, dtype=np.float64)
        g = np.zeros_like(x)
        bad = C.c_int(0)
        e = lib().or_objective_col(self._h, x, y, _ptr(g), None, C.byref(bad), _ptr(col), float(wcol))
        return e, g

    def energy_collision(self, x, col, wcol):
        x = np.ascontiguousarray(x, dtype=np.float64)
        col = np.ascontiguousarray(col, dtype=np.float64)
        g = np.zeros_like(x)
        return lib().or_energy_collision(self._h, x, _ptr(col), float(wcol), _ptr(g)), g

    def internal_energy(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.zeros_like(x)
        return lib().or_internal_energy(self._h, x, _ptr(g)), g

    def first_guess(self, x, v, f):
        y = np.zeros((self.n, 3))
        lib().or_first_guess(self._h, *(np.ascontiguousarray(a, dtype=np.float64) for a in (x, v, f)), y)
        return y

    def residual(self, grad):
        return lib().or_residual(self._h, np.ascontiguousarray(grad, dtype=np.float64))

    def solve(self, x0, y, opts: Opts | None = None):
        x = np.array(x0, dtype=np.float64, order="C")
        st = Stats()
        lib().or_solve(self._h, x, np.ascontiguousarray(y, dtype=np.float64), C.byref(opts or make_opts()), C.byref(st))
        return x, st

    def solve_carry(self, x0, y, pairs=None, opts: Opts | None = None):
        """solve() starting from L-BFGS pairs carried over from an earlier solve.

        pairs: (S, Y) arrays [k, n, 3], the oldest pair first (None or k = 0: an empty
        history).  Returns (x, stats, (S, Y)) with the solve's final pairs, oldest first."""
        o = opts or make_opts()
        M = max(o.lbfgs_m, 1)
        S = np.zeros((M, self.n, 3)); Y = np.zeros((M, self.n, 3))
        k = 0
        if pairs is not None and len(pairs[0]) > 0:
            k = min(len(pairs[0]), o.lbfgs_m)
            S[:k] = pairs[0][-k:]; Y[:k] = pairs[1][-k:]
        cnt = C.c_int(k)
        x = np.array(x0, dtype=np.float64, order="C")
        st = Stats()
        lib().or_solve_carry(self._h, x, np.ascontiguousarray(y, dtype=np.float64), C.byref(o), C.byref(st),
                             S.reshape(-1), Y.reshape(-1), C.byref(cnt))
        return x, st, (S[:cnt.value].copy(), Y[:cnt.value].copy())

    def trajectory(self, x, v, f, steps, opts: Opts | None = None, carry_pairs=True, carry_max_iters=None):
        """steps time steps of one cell along a trajectory with the temporal warm start:
        step 1 starts from y, each later step from y_n + (x_n - y_{n-1}), the previous
        step's converged correction (an addition to the paper's Algorithm 1, which starts
        from y); with carry_pairs each solve also starts from the previous solve's L-BFGS
        pairs, when carry_max_iters is None always, else only while the previous solve
        took at most carry_max_iters iterations.  f: one force [n, 3] or a sequence of
        steps forces.  Returns (x, v, stats of every step)."""
        x = np.array(x, dtype=np.float64); v = np.array(v, dtype=np.float64)
        kappa = float(self.material[MATERIAL_ORDER.index("kappa")])
        corr, pairs, out, last = None, None, [], 0
        for k in range(steps):
            fk = np.asarray(f[k] if np.ndim(f) == 3 else f, dtype=np.float64)
            y = self.first_guess(x, v, fk)
            x0 = y if corr is None else y + corr
            use = carry_pairs and (carry_max_iters is None or last <= carry_max_iters)
            x1, st, p = self.solve_carry(x0, y, pairs if use else None, opts)
            pairs, last = p, st.iterations
            if st.status == 3:  # non-finite: the cell keeps x_n, no correction is kept
                x1 = x.copy()
                corr = np.zeros_like(x)
            else:
                corr = x1 - y
            v = self.post_step(x1, (x1 - x) / self.dt, kappa)
            x = x1
            out.append(st)
        return x, v, out

    def post_step(self, x, v, kappa):
        v = np.array(v, dtype=np.float64, order="C")
        lib().or_post_step(self._h, np.ascontiguousarray(x, dtype=np.float64), v, float(kappa))
        return v

    def step(self, x, v, f, opts: Opts | None = None):
        """One time step of one cell; returns (x_{n+1}, v_{n+1}, stats)."""
        x = np.array(x, dtype=np.float64, order="C")
        v = np.array(v, dtype=np.float64, order="C")
        st = Stats()
        lib().or_step(self._h, x, v, np.ascontiguousarray(f, dtype=np.float64), C.byref(opts or make_opts()), C.byref(st))
        return x, v, st

    def best_rotation(self, y):
        R = np.zeros(9); yc = np.zeros(3); xc = np.zeros(3)
        lib().or_best_rotation(self._h, np.ascontiguousarray(y, dtype=np.float64), R, yc, xc)
        return R.reshape(3, 3), yc, xc

    def ws_features(self, y, f):
        feat = np.zeros((self.n, 9)); R = np.zeros(9)
        lib().or_ws_features(self._h, np.ascontiguousarray(y, dtype=np.float64), np.ascontiguousarray(f, dtype=np.float64), feat, R)
        return feat, R.reshape(3, 3)

    def ws_guess(self, P, x, v, f, bf16_operands=True):
        x1 = np.zeros((self.n, 3))
        lib().or_ws_guess(self._h, np.ascontiguousarray(P, dtype=np.float64), *(np.ascontiguousarray(a, dtype=np.float64) for a in (x, v, f)), x1, int(bf16_operands))
        return x1

    def ws_features_temporal(self, y, f, f_prev, c1, c2):
        """Features of the temporal network at y (trend of the corrections, force change)."""
        a = [np.ascontiguousarray(t, dtype=np.float64) for t in (y, f, f_prev, c1, c2)]
        feat = np.zeros((self.n, 9)); R = np.zeros(9)
        lib().or_ws_features_temporal(self._h, *a, feat, R)
        return feat, R.reshape(3, 3)

    def ws_guess_temporal(self, P, x, v, f, f_prev, c1, c2, bf16_operands=True):
        x1 = np.zeros((self.n, 3))
        a = [np.ascontiguousarray(t, dtype=np.float64) for t in (x, v, f, f_prev, c1, c2)]
        lib().or_ws_guess_temporal(self._h, np.ascontiguousarray(P, dtype=np.float64), *a, x1, int(bf16_operands))
        return x1

    def step_batch(self, x, v, f, opts: Opts | None = None, steps: int = 1, threads: int = 1, col=None, wcol=0.0):
        """steps time steps of every cell of [cells, n, 3] arrays (the same force each
        step); col: optional collision planes [cells, n, 4] with weight wcol."""
        x = np.array(x, dtype=np.float64, order="C")
        v = np.array(v, dtype=np.float64, order="C")
        f = np.ascontiguousarray(f, dtype=np.float64)
        cells = x.shape[0]
        st = (Stats * cells)()
        if col is None:
            lib().or_step_batch(self._h, cells, steps, x, v, f, C.byref(opts or make_opts()), st, threads)
        else:
            col = np.ascontiguousarray(col, dtype=np.float64)
            lib().or_step_batch_col(self._h, cells, steps, x, v, f, C.byref(opts or make_opts()), st, threads,
                                    _ptr(col), float(wcol))
        return x, v, list(st)
