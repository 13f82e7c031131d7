"""Python binding of libpdhg.so (argument marshalling only).

Every step of the solve runs in the library's CUDA kernels; this module only
converts numpy arrays / torch tensors to pointers and back.  If the library
is missing it raises: there is no CPU fallback.

Host arrays (numpy, or CPU tensors) are copied by the library; CUDA tensors
may be passed when the solver is created with ``device_io=True``, in which
case every array argument and output is a device tensor on ``stream``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_lib", "libpdhg.so")

PDHG_OK = 0
PDHG_CONVERGED = 0
PDHG_MAX_ITER = 1
PDHG_NUMERICAL_ERROR = 2
PDHG_TIMEOUT = 3
PDHG_INVALID_ARG = -1
PDHG_CUDA_ERROR = -2
PDHG_OOM = -3
FP64, FP32_MIXED = 0, 1
STATUS_NAMES = {0: "converged", 1: "max_iter", 2: "numerical_error", 3: "timeout",
                -1: "invalid_arg", -2: "cuda_error", -3: "oom"}


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("eval_freq", ctypes.c_int32),
        ("ruiz_iters", ctypes.c_int32),
        ("pock_chambolle", ctypes.c_int32),
        ("eta_safety", ctypes.c_double),
        ("power_max_iter", ctypes.c_int32),
        ("power_rel_tol", ctypes.c_double),
        ("beta_sufficient", ctypes.c_double),
        ("beta_necessary", ctypes.c_double),
        ("beta_artificial", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("io_on_device", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("use_graphs", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("tile_nnz", ctypes.c_int32),
        ("kernel_timing", ctypes.c_int32),
        ("verbose", ctypes.c_int32),
        ("method", ctypes.c_int32),
        ("reflection", ctypes.c_double),
        ("spmv_layout", ctypes.c_int32),
        ("panel_width", ctypes.c_int32),
        ("fp32_screen", ctypes.c_double),
        ("omega_rule", ctypes.c_int32),
        ("pid_kp", ctypes.c_double),
        ("pid_ki", ctypes.c_double),
        ("pid_kd", ctypes.c_double),
        ("persistent", ctypes.c_int32),
        ("wait_limit_ms", ctypes.c_int32),
        ("wait_test", ctypes.c_int32),
        ("step_rule", ctypes.c_int32),
    ]


class PDHGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes)
_SIGS = {
    "pdhg_default_options": (None, [ctypes.POINTER(Options)]),
    "pdhg_create": (_I32, [_PP, _I32, _I32, _P, _P, _P, _P, _P, ctypes.POINTER(Options)]),
    "pdhg_solve": (_I32, [_P, _D, _I64]),
    "pdhg_get": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "pdhg_get_info": (_I32, [_P, _P, _P, _P, _P, _P]),
    "pdhg_warmstart_point": (_I32, [_P, _D, _D, _D, _I32, _P, _P, _P, _P]),
    "pdhg_get_scaling": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "pdhg_get_transpose": (_I32, [_P, _P, _P, _P]),
    "pdhg_get_state": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "pdhg_set_state": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "pdhg_get_log": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "pdhg_get_kernel_timing": (_I32, [_P, _P, _P, _P]),
    "pdhg_get_schedule": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "pdhg_get_layout": (_I32, [_P, _P, _P, _P, _P]),
    "pdhg_get_caches": (_I32, [_P, _P, _P, _P]),
    "pdhg_set_caches": (_I32, [_P, _P, _P, _P]),
    "pdhg_get_kernel_timing_parts": (_I32, [_P, _P, _P]),
    "pdhg_get_launch_count": (_I32, [_P, _P]),
    "pdhg_get_fp64_checks": (_I32, [_P, _P, _P]),
    "pdhg_time_kernels": (_I32, [_P, _I32, _P]),
    "pdhg_get_pid_state": (_I32, [_P, _P, _P]),
    "pdhg_set_pid_state": (_I32, [_P, _D, _D]),
    "pdhg_get_step_state": (_I32, [_P, _P, _P, _P]),
    "pdhg_set_step_state": (_I32, [_P, _D, _D]),
    "pdhg_gather_floor": (_I32, [_P, _I32, _I32, _P]),
    "pdhg_batch_create": (_I32, [_PP, _I32, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Options)]),
    "pdhg_batch_solve": (_I32, [_P, _D, _I64, _P]),
    "pdhg_batch_set_rhs": (_I32, [_P, _P, _P]),
    "pdhg_batch_get": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "pdhg_batch_warmstart_point": (_I32, [_P, _D, _D, _D, _I32, _P, _P, _P, _P]),
    "pdhg_batch_polish": (_I32, [_P, _D, _I32, _P, _P, _P]),
    "pdhg_batch_adjoint": (_I32, [_P, _P, _P, _P, _D, _I32, _P]),
    "pdhg_centered_point_noalloc": (_I32, [_I32, _P, _P, _D, _D, _D, _P, _P, _P, _P]),
    "pdhg_destroy": (None, [_P]),
    "pdhg_last_error": (ctypes.c_char_p, []),
}

_LIB = None


def declared_symbols():
    """Entry points this binding expects the library to export."""
    return list(_SIGS)


def lib(path: Optional[str] = None):
    """Load libpdhg.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIBPATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} not found: build it with paper_2603_03150_gb300.build.build()")
    L = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name, None)
        if f is None:
            continue  # optional entry points are checked by callers
        f.restype = res
        f.argtypes = args
    if path is None:
        _LIB = L
    return L


def _check(status: int, allow_positive: bool = True) -> int:
    if status < 0 or (not allow_positive and status != 0):
        raise PDHGError(status, lib().pdhg_last_error().decode(errors="replace"))
    return status


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """Pointer to a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if _is_torch(a):
        assert a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def centered_point_noalloc(x, z, x_out, z_out, mu_target=None, mu_min: float = 1e-6,
                           delta_max: float = 1e-4, alpha_min: float = 1e-6, stream=None) -> None:
    """Algorithm 1 start point of device vectors (CUDA float64 tensors) into
    caller-provided outputs, with no device allocation by the library."""
    n = int(x.numel())
    _check(lib().pdhg_centered_point_noalloc(n, _ptr(x), _ptr(z), mu_min, delta_max, alpha_min,
                                             _ptr(x_out), _ptr(z_out), _ptr(mu_target), stream),
           allow_positive=False)


class Solver:
    """One LP  min c^T x, Ax = b, x >= 0  held by a library context.

    ``row_ptr``/``col`` int32, ``val``/``b``/``c`` float64.  With
    ``device_io=True`` they (and every output) are CUDA tensors."""

    def __init__(self, m, n, row_ptr, col, val, b, c, precision: str = "fp64",
                 eval_freq: int = 64, ruiz_iters: int = 10, pock_chambolle: bool = True,
                 eta_safety: float = 0.95, power_max_iter: int = 200,
                 power_rel_tol: float = 1e-10, device_io: bool = False, stream=None,
                 use_graphs: bool = True, autotune: bool = True, tile_nnz: int = 0,
                 kernel_timing: bool = False, method: str = "averaged",
                 reflection: float = 1.0, spmv_layout: str = "auto", panel_width: int = 0,
                 fp32_screen: float = 1.0, omega_rule: str = "smooth", pid_kp: float = 0.99,
                 pid_ki: float = 0.01, pid_kd: float = 0.0, wait_limit_ms: int = 1000,
                 wait_test: bool = False, step_rule: str = "constant", verbose: bool = False):
        L = lib()
        o = Options()
        L.pdhg_default_options(ctypes.byref(o))
        o.precision = FP32_MIXED if precision in ("fp32", "fp32_mixed", "mixed") else FP64
        o.eval_freq = eval_freq
        o.ruiz_iters = ruiz_iters
        o.pock_chambolle = 1 if pock_chambolle else 0
        o.eta_safety = eta_safety
        o.power_max_iter = power_max_iter
        o.power_rel_tol = power_rel_tol
        o.io_on_device = 1 if device_io else 0
        o.stream = stream
        o.use_graphs = 1 if use_graphs else 0
        o.autotune = 1 if autotune else 0
        o.tile_nnz = tile_nnz
        o.kernel_timing = 1 if kernel_timing else 0
        if method not in ("averaged", "halpern"):
            raise ValueError("method must be 'averaged' or 'halpern'")
        o.method = 1 if method == "halpern" else 0
        o.reflection = reflection
        layouts = {"auto": 0, "csr": 1, "panels": 2}
        if spmv_layout not in layouts:
            raise ValueError("spmv_layout must be 'auto', 'csr' or 'panels'")
        o.spmv_layout = layouts[spmv_layout]
        o.panel_width = panel_width
        o.fp32_screen = fp32_screen
        if omega_rule not in ("smooth", "pid"):
            raise ValueError("omega_rule must be 'smooth' or 'pid'")
        o.omega_rule = 1 if omega_rule == "pid" else 0
        o.pid_kp, o.pid_ki, o.pid_kd = pid_kp, pid_ki, pid_kd
        o.wait_limit_ms = wait_limit_ms
        o.wait_test = 1 if wait_test else 0
        if step_rule not in ("constant", "adaptive"):
            raise ValueError("step_rule must be 'constant' or 'adaptive'")
        o.step_rule = 1 if step_rule == "adaptive" else 0
        o.verbose = 1 if verbose else 0
        self.m, self.n = int(m), int(n)
        self.device_io = device_io
        self.mixed = o.precision == FP32_MIXED
        if not device_io:
            # host tensors (e.g. pinned torch CPU tensors) pass through as they are
            def host(a, dt):
                return a if _is_torch(a) else np.ascontiguousarray(a, dtype=dt)
            row_ptr, col = host(row_ptr, np.int32), host(col, np.int32)
            val, b, c = host(val, np.float64), host(b, np.float64), host(c, np.float64)
        self._ctx = ctypes.c_void_p()
        self._L = L
        st = L.pdhg_create(ctypes.byref(self._ctx), self.m, self.n, _ptr(row_ptr), _ptr(col),
                           _ptr(val), _ptr(b), _ptr(c), ctypes.byref(o))
        _check(st, allow_positive=False)
        self.status = None

    @classmethod
    def from_lp(cls, lp, **kw):
        return cls(lp.m, lp.n, lp.row_ptr, lp.col, lp.val, lp.b, lp.c, **kw)

    # ------------------------------------------------------------------
    def _new(self, length):
        if self.device_io:
            import torch
            return torch.empty(length, dtype=torch.float64, device="cuda")
        return np.empty(length, dtype=np.float64)

    def solve(self, eps_rel: float = 1e-4, max_iter: int = 1_000_000) -> int:
        self.status = _check(self._L.pdhg_solve(self._ctx, eps_rel, max_iter))
        return self.status

    def get(self, out=None):
        """Returned iterate (x, y, z) and its residual norms; ``out`` may hold
        preallocated (x, y, z) buffers."""
        x, y, z = out if out is not None else (self._new(self.n), self._new(self.m), self._new(self.n))
        rp, rd, gap = _D(), _D(), _D()
        _check(self._L.pdhg_get(self._ctx, _ptr(x), _ptr(y), _ptr(z), ctypes.byref(rp),
                                ctypes.byref(rd), ctypes.byref(gap)))
        return dict(x=x, y=y, z=z, r_P=rp.value, r_D=rd.value, gap=gap.value)

    def info(self, violation: bool = True):
        """Counters; ``violation=False`` skips the float64 report (no GPU work)."""
        it, rs, mv, ca, ls = _I64(), _I64(), _D(), _I32(), _I32()
        _check(self._L.pdhg_get_info(self._ctx, ctypes.byref(it), ctypes.byref(rs),
                                     ctypes.byref(mv) if violation else None,
                                     ctypes.byref(ca), ctypes.byref(ls)))
        return dict(iters=it.value, restarts=rs.value,
                    max_violation=mv.value if violation else None,
                    chosen_average=bool(ca.value), status=ls.value)

    def warmstart_point(self, mu_min: float = 1e-6, delta_max: float = 1e-4,
                        alpha_min: float = 1e-6, unscaled: bool = False, out=None):
        """Algorithm 1 start point (x', y, z') and mu_target."""
        x, y, z = out if out is not None else (self._new(self.n), self._new(self.m), self._new(self.n))
        mu = _D()
        _check(self._L.pdhg_warmstart_point(self._ctx, mu_min, delta_max, alpha_min,
                                            1 if unscaled else 0, _ptr(x), _ptr(y), _ptr(z),
                                            ctypes.byref(mu)))
        return x, y, z, mu.value

    def scaling(self):
        Dr, Dc = self._new(self.m), self._new(self.n)
        smax, eta, om, pit = _D(), _D(), _D(), _I32()
        _check(self._L.pdhg_get_scaling(self._ctx, _ptr(Dr), _ptr(Dc), ctypes.byref(smax),
                                        ctypes.byref(eta), ctypes.byref(om), ctypes.byref(pit)))
        return dict(D_r=Dr, D_c=Dc, sigma_max=smax.value, eta=eta.value, omega0=om.value,
                    power_iters=pit.value)

    def transpose(self, nnz: int):
        rp = np.empty(self.n + 1, dtype=np.int32)
        ci = np.empty(nnz, dtype=np.int32)
        v = np.empty(nnz, dtype=np.float64)
        if self.device_io:
            import torch
            rp, ci, v = (torch.from_numpy(a).cuda() for a in (rp, ci, v))
        _check(self._L.pdhg_get_transpose(self._ctx, _ptr(rp), _ptr(ci), _ptr(v)))
        return rp, ci, v

    def state(self):
        n, m = self.n, self.m
        arrs = [self._new(n), self._new(m), self._new(n), self._new(m), self._new(n), self._new(m)]
        sc = np.empty(8, dtype=np.float64)
        _check(self._L.pdhg_get_state(self._ctx, *[_ptr(a) for a in arrs], _ptr(sc)))
        keys = ["x", "y", "x_avg", "y_avg", "x_last", "y_last"]
        d = dict(zip(keys, arrs))
        caches = [self._new(m), self._new(m), self._new(m)]
        _check(self._L.pdhg_get_caches(self._ctx, *[_ptr(a) for a in caches]))
        d.update(zip(["Ax", "Ax_avg", "Ax_last"], caches))
        d.update(omega=sc[0], k=int(sc[1]), t=int(sc[2]), restarts=int(sc[3]),
                 kkt_last=sc[4], kkt_prev=sc[5], eta=sc[6])
        pi, pe = _D(), _D()
        _check(self._L.pdhg_get_pid_state(self._ctx, ctypes.byref(pi), ctypes.byref(pe)))
        d.update(pid_integral=pi.value, pid_prev=pe.value)
        d.update(self.step_state())
        return d

    def step_state(self):
        """Adaptive step (step_rule 'adaptive'): the next attempt's step, the
        accepted steps since the last restart, the rejected attempts."""
        e, es, rj = _D(), _D(), _I64()
        _check(self._L.pdhg_get_step_state(self._ctx, ctypes.byref(e), ctypes.byref(es),
                                           ctypes.byref(rj)))
        return dict(step_eta=e.value, eta_sum=es.value, step_rejects=rj.value)

    def set_state(self, st):
        sc = np.array([st["omega"], st["k"], st["t"], st["restarts"], st["kkt_last"],
                       st["kkt_prev"], st.get("eta", 0.0), 0.0], dtype=np.float64)
        arrs = [st[k] for k in ["x", "y", "x_avg", "y_avg", "x_last", "y_last"]]
        if not self.device_io:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        _check(self._L.pdhg_set_state(self._ctx, *[_ptr(a) for a in arrs], _ptr(sc)),
               allow_positive=False)
        if "pid_integral" in st:
            _check(self._L.pdhg_set_pid_state(self._ctx, float(st["pid_integral"]),
                                              float(st.get("pid_prev", 0.0))),
                   allow_positive=False)
        if "step_eta" in st and st["step_eta"] > 0:
            _check(self._L.pdhg_set_step_state(self._ctx, float(st["step_eta"]),
                                               float(st.get("eta_sum", 0.0))),
                   allow_positive=False)
        if all(k in st for k in ("Ax", "Ax_avg", "Ax_last")):
            caches = [st[k] for k in ("Ax", "Ax_avg", "Ax_last")]
            if not self.device_io:
                caches = [np.ascontiguousarray(a, dtype=np.float64) for a in caches]
            _check(self._L.pdhg_set_caches(self._ctx, *[_ptr(a) for a in caches]))

    def log(self, cap: int = 4096):
        cnt = _I32()
        k = np.zeros(cap, dtype=np.int64)
        fl = np.zeros(cap, dtype=np.int32)
        kk = np.zeros(3 * cap, dtype=np.float64)
        _check(self._L.pdhg_get_log(self._ctx, cap, ctypes.byref(cnt), _ptr(k), _ptr(fl), _ptr(kk)))
        c = min(cnt.value, cap)
        out = []
        for i in range(c):
            f = int(fl[i])
            out.append(dict(k=int(k[i]), restart=bool(f & 1),
                            cand="average" if f & 2 else "current", r1=bool(f & 4),
                            r2=bool(f & 8), r3=bool(f & 16), kkt_cur=kk[3 * i],
                            kkt_avg=kk[3 * i + 1], omega=kk[3 * i + 2]))
        return out

    def kernel_timing(self):
        a, d, s = _D(), _D(), _I64()
        _check(self._L.pdhg_get_kernel_timing(self._ctx, ctypes.byref(a), ctypes.byref(d),
                                              ctypes.byref(s)))
        return dict(primal_ms=a.value, dual_ms=d.value, samples=s.value)

    def kernel_timing_parts(self):
        """Per kernel: primal SpMV (or fused), primal row pass, dual SpMV (or
        fused), dual row pass (ms; 0 for a fused half-step's row pass)."""
        ms = (ctypes.c_double * 4)()
        s = _I64()
        _check(self._L.pdhg_get_kernel_timing_parts(self._ctx, ms, ctypes.byref(s)))
        return dict(primal_spmv_ms=ms[0], primal_rows_ms=ms[1], dual_spmv_ms=ms[2],
                    dual_rows_ms=ms[3], samples=s.value)

    def schedule(self):
        v = [_I32() for _ in range(8)]
        _check(self._L.pdhg_get_schedule(self._ctx, *[ctypes.byref(x) for x in v]))
        keys = ["a_tile_nnz", "a_block", "a_tiles", "at_tile_nnz", "at_block", "at_tiles",
                "a_variant", "at_variant"]
        return {k: x.value for k, x in zip(keys, v)}

    def layout(self):
        """Column-panel layout per half-step: {"a": {...}, "at": {...}} with the
        panel count (0: CSR tiles), panel width, pseudo-rows and warp tiles."""
        arrs = [(ctypes.c_int64 * 2)() for _ in range(4)]
        _check(self._L.pdhg_get_layout(self._ctx, *arrs))
        keys = ["panels", "panel_width", "pseudo_rows", "tiles"]
        return {side: {k: int(a[j]) for k, a in zip(keys, arrs)} for j, side in enumerate(["a", "at"])}

    def gather_floor(self, on_a: bool, reps: int = 10) -> float:
        """Mean ms of the row-logic-free gather pass over A~ (on_a) or A~^T."""
        ms = _D()
        _check(self._L.pdhg_gather_floor(self._ctx, 1 if on_a else 0, reps, ctypes.byref(ms)))
        return ms.value

    def time_kernels(self, reps: int = 50):
        """Mean ms of back-to-back launches of each half-step on the current
        iterate (state saved and restored): primal, dual, iteration, and the
        panel SpMV kernels alone (0 on CSR tiles)."""
        ms = (ctypes.c_double * 5)()
        _check(self._L.pdhg_time_kernels(self._ctx, reps, ms), allow_positive=False)
        return dict(primal_ms=ms[0], dual_ms=ms[1], iteration_ms=ms[2], primal_spmv_ms=ms[3],
                    dual_spmv_ms=ms[4])

    def fp64_checks(self):
        """Float64 checks of float32-mixed candidates in the last solve:
        (run, rejected)."""
        c, r = _I64(), _I64()
        _check(self._L.pdhg_get_fp64_checks(self._ctx, ctypes.byref(c), ctypes.byref(r)))
        return c.value, r.value

    def launch_count(self) -> int:
        v = _I64()
        _check(self._L.pdhg_get_launch_count(self._ctx, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._L.pdhg_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchSolver(Solver):
    """Many LPs solved together (block-diagonal batch with per-LP state).

    ``lps`` is a list of objects with m, n, row_ptr, col, val, b, c (e.g.
    lpgen.LP); or pass the concatenated arrays via ``arrays=`` (dict with
    m, n, row_ptr, col, val, b, c as the C ABI takes them)."""

    def __init__(self, lps=None, arrays=None, precision: str = "fp64", eval_freq: int = 64,
                 device_io: bool = False, stream=None, use_graphs: bool = True, **kw):
        L = lib()
        o = Options()
        L.pdhg_default_options(ctypes.byref(o))
        o.precision = FP32_MIXED if precision in ("fp32", "fp32_mixed", "mixed") else FP64
        o.eval_freq = eval_freq
        o.io_on_device = 1 if device_io else 0
        o.stream = stream
        o.use_graphs = 1 if use_graphs else 0
        for k, v in kw.items():
            setattr(o, k, v)
        if arrays is None:
            arrays = dict(
                m=np.array([lp.m for lp in lps], dtype=np.int32),
                n=np.array([lp.n for lp in lps], dtype=np.int32),
                row_ptr=np.concatenate([np.asarray(lp.row_ptr, np.int32) for lp in lps]),
                col=np.concatenate([np.asarray(lp.col, np.int32) for lp in lps]),
                val=np.concatenate([np.asarray(lp.val, np.float64) for lp in lps]),
                b=np.concatenate([np.asarray(lp.b, np.float64) for lp in lps]),
                c=np.concatenate([np.asarray(lp.c, np.float64) for lp in lps]))
        self.ms = np.ascontiguousarray(arrays["m"], dtype=np.int32)
        self.ns = np.ascontiguousarray(arrays["n"], dtype=np.int32)
        self.count = int(self.ms.size)
        self.m, self.n = int(self.ms.sum()), int(self.ns.sum())
        self.device_io = device_io
        self.mixed = o.precision == FP32_MIXED
        a = dict(arrays)
        if not device_io:
            for k, dt in [("row_ptr", np.int32), ("col", np.int32), ("val", np.float64),
                          ("b", np.float64), ("c", np.float64)]:
                if not _is_torch(a[k]):
                    a[k] = np.ascontiguousarray(a[k], dtype=dt)
        self._keep = a
        self._ctx = ctypes.c_void_p()
        self._L = L
        st = L.pdhg_batch_create(ctypes.byref(self._ctx), self.count, _ptr(self.ms), _ptr(self.ns),
                                 _ptr(a["row_ptr"]), _ptr(a["col"]), _ptr(a["val"]), _ptr(a["b"]),
                                 _ptr(a["c"]), ctypes.byref(o))
        _check(st, allow_positive=False)
        self.status = None
        self.m_off = np.concatenate([[0], np.cumsum(self.ms)]).astype(np.int64)
        self.n_off = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)

    def set_rhs(self, b, c):
        """New b (float64 [sum m]) and c ([sum n]) for the same A: the scaling,
        transpose, power iteration and schedules are kept; every LP restarts
        from zero."""
        if not self.device_io:
            b = b if _is_torch(b) else np.ascontiguousarray(b, dtype=np.float64)
            c = c if _is_torch(c) else np.ascontiguousarray(c, dtype=np.float64)
        self._keep_rhs = (b, c)
        _check(self._L.pdhg_batch_set_rhs(self._ctx, _ptr(b), _ptr(c)), allow_positive=False)

    def solve(self, eps_rel: float = 1e-4, max_iter: int = 1_000_000):
        st = np.zeros(self.count, dtype=np.int32)
        self.status = _check(self._L.pdhg_batch_solve(self._ctx, eps_rel, max_iter, _ptr(st)))
        self.lp_status = st
        return self.status

    def get(self, out=None):
        x, y, z = out if out is not None else (self._new(self.n), self._new(self.m), self._new(self.n))
        arr = [np.zeros(self.count) for _ in range(4)]
        it = np.zeros(self.count, dtype=np.int64)
        _check(self._L.pdhg_batch_get(self._ctx, _ptr(x), _ptr(y), _ptr(z), *[_ptr(q) for q in arr],
                                      _ptr(it)))
        return dict(x=x, y=y, z=z, r_P=arr[0], r_D=arr[1], gap=arr[2], max_violation=arr[3],
                    iters=it)

    def warmstart_point(self, mu_min: float = 1e-6, delta_max: float = 1e-4,
                        alpha_min: float = 1e-6, unscaled: bool = False, out=None):
        x, y, z = out if out is not None else (self._new(self.n), self._new(self.m), self._new(self.n))
        mu = np.zeros(self.count)
        _check(self._L.pdhg_batch_warmstart_point(self._ctx, mu_min, delta_max, alpha_min,
                                                  1 if unscaled else 0, _ptr(x), _ptr(y), _ptr(z),
                                                  _ptr(mu)))
        return x, y, z, mu

    def split(self, v, side: str):
        """Per-LP pieces of a concatenated vector ('n' or 'm' side)."""
        off = self.n_off if side == "n" else self.m_off
        return [v[off[i]:off[i + 1]] for i in range(self.count)]

    def polish(self, cg_tol: float = 1e-12, cg_max_iter: int = 5000, out=None):
        """Fix the active set B and solve A_B x_B = b in least squares (per LP)."""
        x = out if out is not None else self._new(self.n)
        act = np.zeros(self.count, dtype=np.int32)
        it = np.zeros(self.count, dtype=np.int32)
        _check(self._L.pdhg_batch_polish(self._ctx, cg_tol, cg_max_iter, _ptr(x), _ptr(act),
                                         _ptr(it)))
        return dict(x=x, active=act, cg_iters=it)

    def adjoint(self, grad_x, cg_tol: float = 1e-12, cg_max_iter: int = 5000, out=None):
        """dL/db and dL/dc from dL/dx through the polished solution."""
        gb, gc = out if out is not None else (self._new(self.m), self._new(self.n))
        it = np.zeros(self.count, dtype=np.int32)
        if not self.device_io and not _is_torch(grad_x):
            grad_x = np.ascontiguousarray(grad_x, dtype=np.float64)
        _check(self._L.pdhg_batch_adjoint(self._ctx, _ptr(grad_x), _ptr(gb), _ptr(gc), cg_tol,
                                          cg_max_iter, _ptr(it)))
        return dict(grad_b=gb, grad_c=gc, cg_iters=it)
