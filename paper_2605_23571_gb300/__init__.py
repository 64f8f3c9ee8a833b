"""GB300-native (sm_103a) ensemble-of-4D-Var solver with a randomized spectral
LMP: Python binding of the C ABI in ``include/eda.h`` (``libeda.so``).

The binding only marshals arguments: every step of the path (trajectories,
tangent-linear/adjoint Hessian-vector products, Nystrom approximation, LMP,
batched PCG) runs in the library's CUDA kernels.  There is no CPU fallback:
importing works without a GPU, but creating a handle needs the CUDA library
and a device, and fails loudly otherwise.

Array arguments may be torch tensors (CUDA or CPU) or numpy arrays; they must
be contiguous and FP64 (vectors) or int32 (indices).  Host arrays are staged
by the library through device buffers (see ``include/eda.h``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libeda.so")

EDA_OK, EDA_ERR_INVALID, EDA_ERR_CUDA, EDA_ERR_NUMERIC, EDA_ERR_TIMEOUT, EDA_ERR_STATE = range(6)
EDA_FP64, EDA_MIXED = 0, 1
EDA_THETA_GIVEN, EDA_THETA_LAMBDA_K, EDA_THETA_MID = 0, 1, 2
EDA_CONVERGED, EDA_MAXIT, EDA_NAN, EDA_BREAKDOWN = 0, 1, 2, 3

# every symbol the header declares
EXPORTS = ["eda_version", "eda_last_error", "eda_create", "eda_destroy", "eda_twin",
           "eda_set_trajectory", "eda_sketch", "eda_build_lmp", "eda_set_lmp", "eda_solve_batch", "eda_hvp",
           "eda_bhalf_gaussian", "eda_kernel_launches", "eda_time_hvp_sweep", "eda_autotune",
           "eda_group_create", "eda_group_destroy", "eda_group_last_error", "eda_group_set_trajectories",
           "eda_group_sketch", "eda_group_build_lmp", "eda_group_autotune", "eda_group_solve",
           "eda_ws_create", "eda_ws_destroy", "eda_ws_last_error", "eda_ws_num_params", "eda_ws_set_params",
           "eda_ws_get_params", "eda_ws_set_scales", "eda_ws_get_scales", "eda_ws_loss_grad", "eda_ws_train",
           "eda_ws_infer", "eda_hvp_noalloc", "eda_hvp_noalloc_capacity", "eda_lmp_info",
           "eda_trace", "eda_trace_read", "eda_ws_init", "eda_sweep_plan", "eda_bhalf_apply",
           "eda_plan_tiling", "eda_solve", "eda_lmp_apply", "eda_tail_plans", "eda_set_tail_plan",
           "eda_ritz_lmp"]


class EdaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("eda error %d: %s" % (code, msg))
        self.code = code


class EdaSolveOpts(ctypes.Structure):
    """eda_solve_opts of include/eda.h."""
    _fields_ = [
        ("tol", ctypes.c_double), ("err_tol", ctypes.c_double), ("maxit", ctypes.c_int),
        ("use_lmp", ctypes.c_int), ("split", ctypes.c_int), ("lmp_kind", ctypes.c_int),
        ("x0", ctypes.c_void_p), ("cost_out", ctypes.c_void_p),
    ]


class EdaConfig(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("nsteps", ctypes.c_int), ("F", ctypes.c_double), ("dt", ctypes.c_double),
        ("n_obs_times", ctypes.c_int), ("obs_steps", ctypes.c_void_p), ("obs_ptr", ctypes.c_void_p),
        ("obs_idx", ctypes.c_void_p), ("rinv", ctypes.c_void_p), ("bhalf_w", ctypes.c_int),
        ("bhalf_coef", ctypes.c_void_p), ("n_members", ctypes.c_int), ("ell", ctypes.c_int),
        ("k", ctypes.c_int), ("theta_mode", ctypes.c_int), ("theta", ctypes.c_double),
        ("precision", ctypes.c_int), ("ckpt_every", ctypes.c_int), ("stream", ctypes.c_void_p),
    ]


_lib = None


def build() -> str:
    """Compiles libeda.so in-tree (nvcc, sm_103a)."""
    from . import nvcc_build
    return nvcc_build.build()


def lib() -> ctypes.CDLL:
    """Loads libeda.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libeda.so not built (run paper_2605_23571_gb300.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.eda_version.restype = ctypes.c_char_p
    L.eda_version.argtypes = []
    L.eda_last_error.restype = ctypes.c_char_p
    L.eda_last_error.argtypes = [vp]
    L.eda_create.restype = i
    L.eda_create.argtypes = [ctypes.POINTER(EdaConfig), ctypes.POINTER(vp)]
    L.eda_destroy.restype = i
    L.eda_destroy.argtypes = [vp]
    L.eda_twin.restype = i
    L.eda_twin.argtypes = [vp, vp, i, vp, vp, vp, vp, vp]
    L.eda_set_trajectory.restype = i
    L.eda_set_trajectory.argtypes = [vp, vp, vp, vp]
    L.eda_sketch.restype = i
    L.eda_sketch.argtypes = [vp, vp, i, vp]
    L.eda_build_lmp.restype = i
    L.eda_build_lmp.argtypes = [vp, vp, vp]
    L.eda_set_lmp.restype = i
    L.eda_set_lmp.argtypes = [vp, vp, vp]
    L.eda_trace.restype = i
    L.eda_trace.argtypes = [vp, i]
    L.eda_trace_read.restype = i
    L.eda_trace_read.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(d)]
    L.eda_lmp_info.restype = i
    L.eda_lmp_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d)]
    L.eda_sweep_plan.restype = i
    L.eda_sweep_plan.argtypes = [vp, i, ctypes.POINTER(i)]
    L.eda_bhalf_apply.restype = i
    L.eda_bhalf_apply.argtypes = [vp, i, vp, vp]
    L.eda_plan_tiling.restype = i
    L.eda_plan_tiling.argtypes = [i, i, i, i, i, i, i, i, ctypes.POINTER(i)]
    L.eda_solve_batch.restype = i
    L.eda_solve_batch.argtypes = [vp, d, i, vp, i, vp, vp, vp, vp]
    L.eda_hvp.restype = i
    L.eda_hvp.argtypes = [vp, vp, i, vp, vp, i]
    L.eda_lmp_apply.restype = i
    L.eda_lmp_apply.argtypes = [vp, i, i, i, vp, vp]
    L.eda_tail_plans.restype = i
    L.eda_tail_plans.argtypes = [vp, i, i, ctypes.POINTER(i), vp, vp]
    L.eda_set_tail_plan.restype = i
    L.eda_set_tail_plan.argtypes = [vp, i, i, i, i, i]
    L.eda_ritz_lmp.restype = i
    L.eda_ritz_lmp.argtypes = [vp, i, i, vp, vp]
    L.eda_solve.restype = i
    L.eda_solve.argtypes = [vp, ctypes.POINTER(EdaSolveOpts), vp, vp, vp, vp, vp]
    L.eda_kernel_launches.restype = ctypes.c_longlong
    L.eda_kernel_launches.argtypes = []
    L.eda_autotune.restype = i
    L.eda_autotune.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double)]
    L.eda_time_hvp_sweep.restype = i
    L.eda_time_hvp_sweep.argtypes = [vp, i, i, ctypes.POINTER(ctypes.c_double)]
    L.eda_group_create.restype = i
    L.eda_group_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
    L.eda_group_destroy.restype = i
    L.eda_group_destroy.argtypes = [vp]
    L.eda_group_last_error.restype = ctypes.c_char_p
    L.eda_group_last_error.argtypes = [vp]
    L.eda_group_set_trajectories.restype = i
    L.eda_group_set_trajectories.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.eda_group_sketch.restype = i
    L.eda_group_sketch.argtypes = [vp]
    L.eda_group_build_lmp.restype = i
    L.eda_group_build_lmp.argtypes = [vp]
    L.eda_group_autotune.restype = i
    L.eda_group_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.eda_group_solve.restype = i
    L.eda_group_solve.argtypes = [vp, d, i, i, ctypes.POINTER(vp), vp, vp, vp]
    L.eda_ws_create.restype = i
    L.eda_ws_create.argtypes = [i, i, i, vp, ctypes.POINTER(vp)]
    L.eda_ws_destroy.restype = i
    L.eda_ws_destroy.argtypes = [vp]
    L.eda_ws_last_error.restype = ctypes.c_char_p
    L.eda_ws_last_error.argtypes = [vp]
    L.eda_ws_num_params.restype = ctypes.c_longlong
    L.eda_ws_num_params.argtypes = [vp]
    L.eda_ws_init.restype = i
    L.eda_ws_init.argtypes = [vp, vp]
    L.eda_ws_set_params.restype = i
    L.eda_ws_set_params.argtypes = [vp, vp]
    L.eda_ws_get_params.restype = i
    L.eda_ws_get_params.argtypes = [vp, vp]
    L.eda_ws_set_scales.restype = i
    L.eda_ws_set_scales.argtypes = [vp, d, d]
    L.eda_ws_get_scales.restype = i
    L.eda_ws_get_scales.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.eda_ws_loss_grad.restype = i
    L.eda_ws_loss_grad.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(ctypes.c_double), vp]
    L.eda_ws_train.restype = i
    L.eda_ws_train.argtypes = [vp, vp, vp, vp, i, i, i, d, d, vp, vp]
    L.eda_ws_infer.restype = i
    L.eda_ws_infer.argtypes = [vp, vp, vp, i, vp]
    L.eda_hvp_noalloc.restype = i
    L.eda_hvp_noalloc.argtypes = [vp, vp, i, vp, vp, i]
    L.eda_hvp_noalloc_capacity.restype = ctypes.c_longlong
    L.eda_hvp_noalloc_capacity.argtypes = [i]
    L.eda_bhalf_gaussian.restype = i
    L.eda_bhalf_gaussian.argtypes = [i, d, d, vp, i, ctypes.POINTER(ctypes.c_int)]
    _lib = L
    return L


def _ptr(a, dtype, count: Optional[int] = None, name: str = "array"):
    """Address of a contiguous torch tensor or numpy array of the given dtype."""
    return _ptr_impl(a, dtype, count, name)


def _ptr_impl(a, dtype, count, name):
    """Address of a contiguous torch tensor or numpy array of the given dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("%s must be a contiguous %s numpy array" % (name, np.dtype(dtype)))
        if count is not None and a.size < count:
            raise ValueError("%s has %d elements, needs %d" % (name, a.size, count))
        return a.ctypes.data
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[np.dtype(dtype).type]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError("%s must be a contiguous %s tensor" % (name, tdt))
        if count is not None and a.numel() < count:
            raise ValueError("%s has %d elements, needs %d" % (name, a.numel(), count))
        return a.data_ptr()
    raise TypeError("%s must be a numpy array or torch tensor" % name)


PLAN_KINDS = ("cluster", "multi-launch", "warp")
PLAN_KEYS = ("kind", "ctas_per_vector", "threads", "C", "K", "halo", "owned", "smem")


def plan_tiling(n, fp64, w, kind, cs=0, threads=0, K=8, C=0, ckpt=False):
    """The sweep tiling the library would use (host only, no GPU): kind
    'cluster' (cs CTAs per vector), 'multi-launch' (`threads` per CTA; with
    ckpt, for a trajectory checkpointed every K steps) or 'warp'; a dict as
    Handle.eda_sweep_plan returns, or None if it does not fit."""
    info = (ctypes.c_int * 8)()
    k = 3 if (ckpt and kind == "multi-launch") else PLAN_KINDS.index(kind)
    rc = lib().eda_plan_tiling(int(n), int(bool(fp64)), int(w), k, int(cs), int(threads), int(K), int(C), info)
    if rc != EDA_OK:
        return None
    out = dict(zip(PLAN_KEYS, list(info)))
    out["kind"] = PLAN_KINDS[out["kind"]]
    return out


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().eda_kernel_launches())


def bhalf_gaussian(n: int, length_scale: float, sigma_b: float = 1.0) -> np.ndarray:
    """Taps of U_B for a Gaussian correlation of length L (library host helper)."""
    L = lib()
    cap = n // 2 + 2
    out = np.zeros(cap)
    w = ctypes.c_int(0)
    rc = L.eda_bhalf_gaussian(int(n), float(length_scale), float(sigma_b), out.ctypes.data, cap,
                              ctypes.byref(w))
    if rc != EDA_OK:
        raise EdaError(rc, L.eda_last_error(None).decode())
    return out[: w.value + 1].copy()


class Handle:
    """One EDA problem on the current CUDA device (wraps ``eda_handle``).

    Methods carry the C names and arguments of ``include/eda.h``.
    """

    def __init__(self, n, nsteps, obs_steps, obs_ptr, obs_idx, rinv, bhalf_coef, n_members,
                 ell, k, theta_mode=EDA_THETA_MID, theta=1.0, precision=EDA_FP64, ckpt_every=0,
                 F=8.0, dt=0.025, stream=None):
        self._L = lib()
        self.n, self.nsteps, self.M = int(n), int(nsteps), int(n_members)
        self._keep = [np.ascontiguousarray(obs_steps, dtype=np.int32),
                      np.ascontiguousarray(obs_ptr, dtype=np.int32),
                      np.ascontiguousarray(obs_idx, dtype=np.int32),
                      np.ascontiguousarray(rinv, dtype=np.float64),
                      np.ascontiguousarray(bhalf_coef, dtype=np.float64)]
        steps, ptr, idx, rv, coef = self._keep
        self.p = int(ptr[-1])
        self.ell, self.k = int(ell), int(k)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:  # pragma: no cover
                stream = 0
        cfg = EdaConfig(n=self.n, nsteps=self.nsteps, F=float(F), dt=float(dt),
                        n_obs_times=len(steps), obs_steps=steps.ctypes.data,
                        obs_ptr=ptr.ctypes.data, obs_idx=idx.ctypes.data, rinv=rv.ctypes.data,
                        bhalf_w=len(coef) - 1, bhalf_coef=coef.ctypes.data, n_members=self.M,
                        ell=self.ell, k=self.k, theta_mode=int(theta_mode), theta=float(theta),
                        precision=int(precision), ckpt_every=int(ckpt_every),
                        stream=ctypes.c_void_p(int(stream)))
        h = ctypes.c_void_p(None)
        rc = self._L.eda_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != EDA_OK:
            raise EdaError(rc, self._L.eda_last_error(None).decode())
        self._h = h

    @classmethod
    def from_spec(cls, spec, taps, precision=EDA_FP64, stream=None, **kw):
        args = dict(n=spec.n, nsteps=spec.nsteps, obs_steps=spec.obs_steps, obs_ptr=spec.obs_ptr,
                    obs_idx=spec.obs_idx, rinv=spec.rinv, bhalf_coef=taps,
                    n_members=spec.n_members, ell=spec.ell, k=spec.k, theta_mode=spec.theta_mode,
                    theta=spec.theta, precision=precision, ckpt_every=spec.ckpt_every, F=spec.F,
                    dt=spec.dt, stream=stream)
        args.update(kw)
        return cls(**args)

    def _check(self, rc):
        if rc != EDA_OK:
            raise EdaError(rc, self._L.eda_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.eda_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ----------------------------------------------------------------- calls
    def eda_twin(self, x_spin0, spinup, eta_b, eta_o, xb_out, y_out, xt0_out=None):
        n, M, p = self.n, self.M, self.p
        self._check(self._L.eda_twin(
            self._h, _ptr(x_spin0, np.float64, n, "x_spin0"), int(spinup),
            _ptr(eta_b, np.float64, M * n, "eta_b"), _ptr(eta_o, np.float64, M * p, "eta_o"),
            _ptr(xb_out, np.float64, M * n, "xb_out"), _ptr(y_out, np.float64, M * p, "y_out"),
            _ptr(xt0_out, np.float64, n, "xt0_out")))

    def eda_set_trajectory(self, xb, y, rhs_out=None):
        n, M, p = self.n, self.M, self.p
        self._check(self._L.eda_set_trajectory(
            self._h, _ptr(xb, np.float64, M * n, "xb"), _ptr(y, np.float64, M * p, "y"),
            _ptr(rhs_out, np.float64, M * n, "rhs_out")))

    def eda_sketch(self, phi=None, q=1, y_out=None):
        n, ell = self.n, self.ell
        self._check(self._L.eda_sketch(self._h, _ptr(phi, np.float64, ell * n, "phi"), int(q),
                                       _ptr(y_out, np.float64, ell * n, "y_out")))

    def eda_build_lmp(self, eigvals_out=None, s_out=None):
        self._check(self._L.eda_build_lmp(self._h, _ptr(eigvals_out, np.float64, self.k, "eigvals_out"),
                                          _ptr(s_out, np.float64, self.k * self.n, "s_out")))

    def eda_set_lmp(self, s_in, eigvals_in):
        self._check(self._L.eda_set_lmp(self._h, _ptr(s_in, np.float64, self.k * self.n, "s_in"),
                                        _ptr(eigvals_in, np.float64, self.k, "eigvals_in")))

    def eda_trace(self, enable=True, every=1):
        """Starts (enable, tracing one sweep in `every`) or stops the sweep
        trace of this handle."""
        self._check(self._L.eda_trace(self._h, int(every) if enable else 0))

    def eda_trace_read(self, fp64=False):
        """(sweeps, columns, ms) recorded for the FP64 or the FP32 sweeps."""
        a, b, c = ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_double(0.0)
        self._check(self._L.eda_trace_read(self._h, 1 if fp64 else 0, ctypes.byref(a), ctypes.byref(b),
                                           ctypes.byref(c)))
        return a.value, b.value, c.value

    def eda_lmp_info(self):
        """(path, rank, shift) of the current LMP: path 0 Cholesky, 1 shift,
        2 truncated eigendecomposition; rank = informative modes."""
        path, rank, shift = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self._L.eda_lmp_info(self._h, ctypes.byref(path), ctypes.byref(rank), ctypes.byref(shift)))
        return path.value, rank.value, shift.value


    def eda_sweep_plan(self, fp64=False):
        """The tiling of the FP64 or FP32 Hessian-product sweeps as a dict
        (kind: cluster, multi-launch or warp; C values per thread, halo
        refresh period K, ...)."""
        info = (ctypes.c_int * 8)()
        self._check(self._L.eda_sweep_plan(self._h, int(bool(fp64)), info))
        out = dict(zip(PLAN_KEYS, list(info)))
        out["kind"] = PLAN_KINDS[out["kind"]]
        return out

    def eda_ritz_lmp(self, member=0, iters=None, b=None):
        """Installs the LMP of the k leading Ritz pairs from `iters` CG
        iterations (default k) on member's Hessian, right-hand side b [n]
        (default the member's own); returns all Ritz values (descending)."""
        iters = self.k if iters is None else int(iters)
        out = np.zeros(iters)
        self._check(self._L.eda_ritz_lmp(self._h, int(member), iters, _ptr(b, np.float64, self.n, "b"),
                                         out.ctypes.data))
        return out

    def eda_tail_plans(self, fp64=True):
        """The convergence tail's tilings of the persistent PCG: a list of
        (level, plan dict), levels decreasing."""
        cnt = ctypes.c_int(0)
        self._check(self._L.eda_tail_plans(self._h, int(bool(fp64)), 0, ctypes.byref(cnt), None, None))
        k = cnt.value
        lev = (ctypes.c_int * max(1, k))()
        info = (ctypes.c_int * max(8, 8 * k))()
        self._check(self._L.eda_tail_plans(self._h, int(bool(fp64)), k, ctypes.byref(cnt), lev, info))
        out = []
        for i in range(k):
            d = dict(zip(PLAN_KEYS, list(info[8 * i:8 * i + 8])))
            d["kind"] = PLAN_KINDS[d["kind"]]
            out.append((int(lev[i]), d))
        return out

    def eda_set_tail_plan(self, level, cs=0, K=0, C=0, fp64=True):
        """Installs the cluster tiling of cs CTAs (refresh K) for at most
        `level` active members; level 0 removes every tail tiling."""
        self._check(self._L.eda_set_tail_plan(self._h, int(bool(fp64)), int(level), int(cs), int(K), int(C)))

    def eda_solve_batch(self, tol, maxit, x0, use_lmp, dz_out, iters_out=None, relres_out=None,
                        status_out=None):
        n, M = self.n, self.M
        self._check(self._L.eda_solve_batch(
            self._h, float(tol), int(maxit), _ptr(x0, np.float64, M * n, "x0"), 1 if use_lmp else 0,
            _ptr(dz_out, np.float64, M * n, "dz_out"), _ptr(iters_out, np.int32, M, "iters_out"),
            _ptr(relres_out, np.float64, M, "relres_out"), _ptr(status_out, np.int32, M, "status_out")))

    def eda_solve(self, dz_out, tol=0.0, err_tol=0.0, maxit=100, use_lmp=True, split=False, lmp_kind=0,
                  x0=None, cost_out=None, iters_out=None, relres_out=None, err_bound_out=None, status_out=None):
        """Batched PCG with the options of eda_solve_opts (certified error
        stopping err_tol, cost record cost_out [(L+1) x (maxit+1)])."""
        n, M = self.n, self.M
        o = EdaSolveOpts(float(tol), float(err_tol), int(maxit), 1 if use_lmp else 0, 1 if split else 0,
                         int(lmp_kind), _ptr(x0, np.float64, M * n, "x0"),
                         _ptr(cost_out, np.float64, M * (int(maxit) + 1), "cost_out"))
        self._check(self._L.eda_solve(
            self._h, ctypes.byref(o), _ptr(dz_out, np.float64, M * n, "dz_out"),
            _ptr(iters_out, np.int32, M, "iters_out"), _ptr(relres_out, np.float64, M, "relres_out"),
            _ptr(err_bound_out, np.float64, M, "err_bound_out"), _ptr(status_out, np.int32, M, "status_out")))

    def eda_lmp_apply(self, R, Z, which=0, kind=0):
        """Z = R + S diag(coef) S^T R for every row of R: which 0 P_theta,
        1 U_theta, 2 U_theta^{-1}; kind 0 CUDA cores, 1 tensor cores."""
        ncol = int(R.shape[0])
        self._check(self._L.eda_lmp_apply(self._h, int(which), int(kind), ncol,
                                          _ptr(R, np.float64, ncol * self.n, "R"),
                                          _ptr(Z, np.float64, ncol * self.n, "Z")))

    def eda_autotune(self, which=0):
        """Times the sweep tilings on the stored trajectories, keeps the fastest."""
        ms = ctypes.c_double(0.0)
        self._check(self._L.eda_autotune(self._h, int(which), ctypes.byref(ms)))
        return ms.value

    def eda_hvp_noalloc(self, member_of_col, V, HV, include_identity=True):
        """eda_hvp without any device allocation (device arguments only, the
        observation stash in the library's fixed scratch array)."""
        ncol = int(member_of_col.shape[0])
        n = self.n
        self._check(self._L.eda_hvp_noalloc(self._h, _ptr(member_of_col, np.int32, ncol, "member_of_col"), ncol,
                                            _ptr(V, np.float64, ncol * n, "V"),
                                            _ptr(HV, np.float64, ncol * n, "HV"), 1 if include_identity else 0))

    def eda_time_hvp_sweep(self, reps=10, fp64=False):
        """Mean milliseconds per launch of the batched member HVP sweep."""
        ms = ctypes.c_double(0.0)
        self._check(self._L.eda_time_hvp_sweep(self._h, int(reps), 1 if fp64 else 0, ctypes.byref(ms)))
        return ms.value

    def eda_bhalf_apply(self, V, OUT):
        """OUT[c] = U_B V[c] (control-variable transform) for every row of V."""
        ncol = int(V.shape[0])
        self._check(self._L.eda_bhalf_apply(self._h, ncol, _ptr(V, np.float64, ncol * self.n, "V"),
                                            _ptr(OUT, np.float64, ncol * self.n, "OUT")))

    def eda_hvp(self, member_of_col, V, HV, include_identity=True):
        ncol = int(np.asarray(member_of_col.shape[0] if hasattr(member_of_col, "shape") else len(member_of_col)))
        n = self.n
        self._check(self._L.eda_hvp(self._h, _ptr(member_of_col, np.int32, ncol, "member_of_col"), ncol,
                                    _ptr(V, np.float64, ncol * n, "V"), _ptr(HV, np.float64, ncol * n, "HV"),
                                    1 if include_identity else 0))


class Group:
    """Independent EDA problems solved together (wraps ``eda_group``).

    ``handles`` are ``Handle`` objects of one precision and stream; they must
    outlive the group.  Methods carry the C names of ``include/eda.h``.
    """

    def __init__(self, handles):
        self._L = lib()
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        g = ctypes.c_void_p(None)
        rc = self._L.eda_group_create(arr, len(self.handles), ctypes.byref(g))
        if rc != EDA_OK:
            raise EdaError(rc, self._L.eda_last_error(None).decode())
        self._g = g
        self.total_members = sum(h.M for h in self.handles)

    def _check(self, rc):
        if rc != EDA_OK:
            raise EdaError(rc, self._L.eda_group_last_error(self._g).decode())

    def close(self):
        if getattr(self, "_g", None) is not None and self._g.value:
            self._L.eda_group_destroy(self._g)
            self._g = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def eda_group_set_trajectories(self, xbs, ys):
        xa = (ctypes.c_void_p * len(xbs))(*[_ptr(x, np.float64, h.M * h.n, "xb")
                                            for x, h in zip(xbs, self.handles)])
        ya = (ctypes.c_void_p * len(ys))(*[_ptr(y, np.float64, h.M * h.p, "y")
                                           for y, h in zip(ys, self.handles)])
        self._check(self._L.eda_group_set_trajectories(self._g, xa, ya))

    def eda_group_sketch(self):
        self._check(self._L.eda_group_sketch(self._g))

    def eda_group_build_lmp(self):
        self._check(self._L.eda_group_build_lmp(self._g))

    def eda_group_autotune(self):
        ms = ctypes.c_double(0.0)
        self._check(self._L.eda_group_autotune(self._g, ctypes.byref(ms)))
        return ms.value

    def eda_group_solve(self, tol, maxit, use_lmp, dz_outs=None, iters_out=None, relres_out=None,
                        status_out=None):
        T = self.total_members
        da = None
        if dz_outs is not None:
            da = (ctypes.c_void_p * len(dz_outs))(*[_ptr(z, np.float64, h.M * h.n, "dz")
                                                    for z, h in zip(dz_outs, self.handles)])
        self._check(self._L.eda_group_solve(self._g, float(tol), int(maxit), 1 if use_lmp else 0, da,
                                            _ptr(iters_out, np.int32, T, "iters_out"),
                                            _ptr(relres_out, np.float64, T, "relres_out"),
                                            _ptr(status_out, np.int32, T, "status_out")))


class WarmStart:
    """The learned warm-start network (wraps ``eda_ws``); methods carry the C
    names of ``include/eda.h``."""

    def __init__(self, n, hidden=64, max_batch=64, stream=None):
        self._L = lib()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:  # pragma: no cover
                stream = 0
        w = ctypes.c_void_p(None)
        rc = self._L.eda_ws_create(int(n), int(hidden), int(max_batch), ctypes.c_void_p(int(stream)),
                                   ctypes.byref(w))
        if rc != EDA_OK:
            raise EdaError(rc, self._L.eda_last_error(None).decode())
        self._w = w
        self.n, self.hidden, self.max_batch = int(n), int(hidden), int(max_batch)
        self.num_params = int(self._L.eda_ws_num_params(w))

    def _check(self, rc):
        if rc != EDA_OK:
            raise EdaError(rc, self._L.eda_ws_last_error(self._w).decode())

    def close(self):
        if getattr(self, "_w", None) is not None and self._w.value:
            self._L.eda_ws_destroy(self._w)
            self._w = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def eda_ws_init(self, draws):
        """He initialisation from num_params standard-normal draws (FP64)."""
        self._check(self._L.eda_ws_init(self._w, _ptr(draws, np.float64, self.num_params, "draws")))

    def eda_ws_set_params(self, params):
        self._check(self._L.eda_ws_set_params(self._w, _ptr(params, np.float32, self.num_params, "params")))

    def eda_ws_get_params(self):
        out = np.zeros(self.num_params, dtype=np.float32)
        self._check(self._L.eda_ws_get_params(self._w, out.ctypes.data))
        return out

    def eda_ws_set_scales(self, s_b, s_z):
        self._check(self._L.eda_ws_set_scales(self._w, float(s_b), float(s_z)))

    def eda_ws_get_scales(self):
        a, b = ctypes.c_double(0), ctypes.c_double(0)
        self._check(self._L.eda_ws_get_scales(self._w, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def eda_ws_loss_grad(self, rhs, ctrl, sol):
        count = int(rhs.shape[0])
        loss = ctypes.c_double(0.0)
        grad = np.zeros(self.num_params, dtype=np.float32)
        n = self.n
        self._check(self._L.eda_ws_loss_grad(self._w, _ptr(rhs, np.float64, count * n, "rhs"),
                                             _ptr(ctrl, np.float64, count * n, "ctrl"),
                                             _ptr(sol, np.float64, count * n, "sol"), count,
                                             ctypes.byref(loss), grad.ctypes.data))
        return loss.value, grad

    def eda_ws_train(self, rhs, ctrl, sol, epochs, batch, lr, weight_decay=0.0, order=None):
        count = int(rhs.shape[0])
        n = self.n
        losses = np.zeros(max(epochs, 1))
        self._check(self._L.eda_ws_train(self._w, _ptr(rhs, np.float64, count * n, "rhs"),
                                         _ptr(ctrl, np.float64, count * n, "ctrl"),
                                         _ptr(sol, np.float64, count * n, "sol"), count, int(epochs),
                                         int(batch), float(lr), float(weight_decay),
                                         _ptr(order, np.int32, epochs * count, "order"), losses.ctypes.data))
        return losses[:epochs]

    def eda_ws_infer(self, rhs, ctrl, out):
        count = int(rhs.shape[0])
        n = self.n
        self._check(self._L.eda_ws_infer(self._w, _ptr(rhs, np.float64, count * n, "rhs"),
                                         _ptr(ctrl, np.float64, count * n, "ctrl"), count,
                                         _ptr(out, np.float64, count * n, "out")))
