"""Thin Python binding of the acac C ABI (include/acac.h).

Argument marshalling only: every step of the solve runs in libacac.so's CUDA
kernels.  Device arrays are torch CUDA tensors (contiguous float64 state vectors /
fields, or Krylov-precision tensors where the C ABI takes void*); the handle
enqueues all work on the torch stream that is current when it is created.

The library must have been built (paper_2007_04560_gb300.build.build()); loading
fails loudly otherwise — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libacac.so")

OK = 0
E_ARG = -1
E_CUDA = -2
E_DOMAIN = -3
E_DIVERGED = -4
E_DT_UNDERFLOW = -5
E_TIMEOUT = -6
E_NOMEM = -7


class AcacError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = _lib().acac_status_string(status).decode() if _LIB is not None else str(status)
        super().__init__("%s: %s (%d)" % (where or "acac", msg, status))


class acac_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3), ("bc", ctypes.c_int),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("theta", ctypes.c_double),
        ("gamma", ctypes.c_double), ("rho", ctypes.c_double), ("taylor_S", ctypes.c_int),
        ("dt_mode", ctypes.c_int), ("dt0", ctypes.c_double), ("dt_min", ctypes.c_double),
        ("dt_max", ctypes.c_double), ("eta0", ctypes.c_double),
        ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
        ("gmres_rtol", ctypes.c_double), ("gmres_atol", ctypes.c_double), ("gmres_restart", ctypes.c_int),
        ("gmres_maxit", ctypes.c_int), ("ras_parts", ctypes.c_int * 3), ("ras_overlap", ctypes.c_int),
        ("ras_type", ctypes.c_int), ("ilu_reuse", ctypes.c_int), ("precision", ctypes.c_int),
        ("jac_mode", ctypes.c_int), ("batch", ctypes.c_int), ("cgs_refine", ctypes.c_int),
        ("graphs", ctypes.c_int), ("ras_window", ctypes.c_int), ("subdomain_solver", ctypes.c_int),
    ]


class acac_step_info(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("dt", ctypes.c_double), ("eta", ctypes.c_double),
        ("energy", ctypes.c_double), ("mass", ctypes.c_double), ("fnorm0", ctypes.c_double),
        ("fnorm", ctypes.c_double), ("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int),
        ("divergences", ctypes.c_int), ("status", ctypes.c_int), ("line_search_cuts", ctypes.c_int),
        ("ilu_factorizations", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every symbol declared in include/acac.h, with its ctypes signature.
_P = ctypes.c_void_p
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)
SIGNATURES = {
    "acac_default_params": (None, [ctypes.POINTER(acac_params)]),
    "acac_create": (ctypes.c_int, [ctypes.POINTER(acac_params), _P, ctypes.POINTER(_P)]),
    "acac_step": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(acac_step_info)]),
    "acac_step_host": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(acac_step_info)]),
    "acac_energy": (ctypes.c_int, [_P, _P, _P, _PD, _PD]),
    "acac_destroy": (None, [_P]),
    "acac_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "acac_residual": (ctypes.c_int, [_P, _P, _P, _D, _P, _PD]),
    "acac_jacobian": (ctypes.c_int, [_P, _P, _P, _D, _P]),
    "acac_spmv": (ctypes.c_int, [_P, _P, _P, _P]),
    "acac_jvp": (ctypes.c_int, [_P, _P, _P, _D, _P, _P]),
    "acac_ras_factor": (ctypes.c_int, [_P, _P]),
    "acac_ras_apply": (ctypes.c_int, [_P, _P, _P]),
    "acac_gmres": (ctypes.c_int, [_P, _P, _P, _D, _P, _P, _PI, _PD]),
    "acac_nks_solve": (ctypes.c_int, [_P, _P, _D, _P, ctypes.POINTER(acac_step_info)]),
    "acac_residual_noalloc": (ctypes.c_int, [ctypes.POINTER(acac_params), _P, _P, _D, _P, _PD, _P]),
    "acac_log": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
    "acac_peak_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _PD, _PD, _P]),
    "acac_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "acac_profile_mask": (ctypes.c_int, [_P, ctypes.c_uint]),
    "acac_wait_selftest": (ctypes.c_int, [_P, ctypes.c_int]),
    "acac_subdomain_pattern": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              _PI, _PI, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    "acac_kernel_stats": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _PD, _PD, _PD]),
    "acac_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "acac_set_coeffs": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _D, _D, _D]),
    "acac_autotune": (ctypes.c_int, [ctypes.POINTER(acac_params), _P, _P, ctypes.c_int, _P,
                                     ctypes.POINTER(acac_params), _PD, _PI]),
    "acac_jacobian_x0": (ctypes.c_int, [_P, _P, _P, _D, _P]),
    "acac_spmv_t": (ctypes.c_int, [_P, _P, _P, _P]),
    "acac_loss": (ctypes.c_int, [_P, _P, _P, _D, _D, _PD, _P, _PD]),
    "acac_adjoint_step": (ctypes.c_int, [_P, _P, _P, _D, _P, _P, _PD, _D, _PI]),
    "acac_adjoint": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _D, ctypes.c_int, _P, _P, _D, _D, _D, _PD, _P, _P,
                                    _PD, _PI]),
}

NKERNEL = 14

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libacac.so is not built (run paper_2007_04560_gb300.build.build()); "
                               "there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def load():
    """Load libacac.so (raises if it is missing) and return the ctypes handle."""
    return _lib()


def _check(st, where):
    if st != OK:
        raise AcacError(st, where)


def to_c_params(p) -> acac_params:
    """Marshal a workloads.Params (or any object with the same fields) into acac_params."""
    c = acac_params()
    _lib().acac_default_params(ctypes.byref(c))
    for name, ctype in acac_params._fields_:
        if not hasattr(p, name):
            continue
        val = getattr(p, name)
        if name in ("n", "ras_parts"):
            setattr(c, name, (ctypes.c_int * 3)(*[int(x) for x in val]))
        elif name == "L":
            setattr(c, name, (ctypes.c_double * 3)(*[float(x) for x in val]))
        else:
            setattr(c, name, val)
    return c


def _dev(t, dtype=None, numel=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements" % (name, numel))
    return ctypes.c_void_p(t.data_ptr())


def acac_create(p, stream=None):
    """acac_create on the current torch CUDA stream (or the given one)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    h = ctypes.c_void_p()
    cp = to_c_params(p)
    _check(_lib().acac_create(ctypes.byref(cp), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)),
           "acac_create")
    return h


def acac_destroy(h):
    _lib().acac_destroy(h)


def acac_status_string(status: int) -> str:
    return _lib().acac_status_string(status).decode()


def acac_residual_noalloc(p, X1, X0, dt, F, stream=None, check=True):
    """F(X1) without a handle and without device allocation (grids up to 512x512 cells).
    X1, X0 and F must be on the current CUDA device.  Returns (status, ||F||)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    n = 2 * int(p.n[0]) * int(p.n[1]) * (int(p.n[2]) if p.dim == 3 else 1)
    cur = torch.cuda.current_device()
    for name, t in (("X1", X1), ("X0", X0), ("F", F)):
        if isinstance(t, torch.Tensor) and t.is_cuda and t.device.index != cur:
            raise ValueError("%s is on cuda:%d; acac_residual_noalloc runs on the current device cuda:%d"
                             % (name, t.device.index, cur))
    cp = to_c_params(p)
    fn = ctypes.c_double()
    st = _lib().acac_residual_noalloc(ctypes.byref(cp), _dev(X1, torch.float64, n, "X1"),
                                      _dev(X0, torch.float64, n, "X0"), float(dt), _dev(F, torch.float64, n, "F"),
                                      ctypes.byref(fn), ctypes.c_void_p(stream.cuda_stream))
    if check:
        _check(st, "acac_residual_noalloc")
    return st, fn.value


def acac_log(x, y, stream=None):
    """y = ln x with the library's device logarithm (float64 CUDA tensors)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(_lib().acac_log(_dev(x, torch.float64, None, "x"), _dev(y, torch.float64, x.numel(), "y"),
                           x.numel(), ctypes.c_void_p(stream.cuda_stream)), "acac_log")


def acac_peak_probe(kind, iters, stream=None):
    """Measured multiply-add rate of the current device: kind 0 double, 1 float.
    Returns (TFLOP/s, ms of the timed launch)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib().acac_peak_probe(int(kind), int(iters), ctypes.byref(tf), ctypes.byref(ms),
                                  ctypes.c_void_p(stream.cuda_stream)), "acac_peak_probe")
    return tf.value, ms.value


def acac_subdomain_pattern(dim, W, H, D, solver):
    """(ptr, col) numpy arrays of the block pattern of a subdomain factorization with fill
    (host only; see include/acac.h)."""
    import numpy as np
    n = W * H * (D if dim == 3 else 1)
    nnz = ctypes.c_longlong(0)
    st = _lib().acac_subdomain_pattern(dim, W, H, D, solver, None, None, 0, ctypes.byref(nnz))
    if nnz.value == 0:
        _check(st, "acac_subdomain_pattern")
    ptr = np.zeros(n + 1, dtype=np.int32)
    col = np.zeros(max(1, nnz.value), dtype=np.int32)
    _check(_lib().acac_subdomain_pattern(dim, W, H, D, solver, ptr.ctypes.data_as(_PI), col.ctypes.data_as(_PI),
                                         nnz.value, ctypes.byref(nnz)), "acac_subdomain_pattern")
    return ptr, col[:nnz.value]


def acac_autotune(p, u, v, trial_steps=3, stream=None):
    """Fastest Schwarz partition for the problem p (a workloads.Params) from the state
    (u, v) (float64 CUDA tensors, not modified).  Returns (params, ms_per_step,
    ncandidates) with params a copy of p with ras_parts / ras_overlap replaced."""
    import dataclasses

    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    n = int(p.n[0]) * int(p.n[1]) * (int(p.n[2]) if p.dim == 3 else 1) * int(getattr(p, "batch", 1))
    cp = to_c_params(p)
    best = acac_params()
    ms, nc = ctypes.c_double(), ctypes.c_int()
    _check(_lib().acac_autotune(ctypes.byref(cp), _dev(u, torch.float64, n, "u"), _dev(v, torch.float64, n, "v"),
                                int(trial_steps), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(best),
                                ctypes.byref(ms), ctypes.byref(nc)), "acac_autotune")
    out = dataclasses.replace(p, ras_parts=tuple(best.ras_parts), ras_overlap=best.ras_overlap)
    return out, ms.value, nc.value


class Solver:
    """Owns one acac handle.  Method names follow the C ABI without the prefix.

    With params.batch = B > 1 the handle is an ensemble: step / step_host / energy
    take the B members' fields one after another (B*N values per field) and return
    one report (or energy, mass) per member."""

    def __init__(self, params, stream=None):
        import torch
        self.params = params
        self.B = int(getattr(params, "batch", 1))
        self.N = int(params.n[0]) * int(params.n[1]) * (int(params.n[2]) if params.dim == 3 else 1)
        self.kdtype = torch.float32 if params.precision == 1 else torch.float64
        self.nslot = 13 if params.dim == 2 else 25
        self.h = acac_create(params, stream)

    def close(self):
        if self.h:
            acac_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- time stepping
    def _infos(self):
        return (acac_step_info * self.B)()

    def _out(self, infos):
        return infos[0] if self.B == 1 else list(infos)

    def step(self, u, v, check=True):
        """One accepted step in place; returns the report (a list of B for an ensemble)."""
        import torch
        infos = self._infos()
        nb = self.B * self.N
        st = _lib().acac_step(self.h, _dev(u, torch.float64, nb, "u"), _dev(v, torch.float64, nb, "v"), infos)
        if check:
            _check(st, "acac_step")
        return self._out(infos)

    def set_coeffs(self, member, alpha, beta, theta, gamma, rho):
        _check(_lib().acac_set_coeffs(self.h, int(member), float(alpha), float(beta), float(theta), float(gamma),
                                      float(rho)), "acac_set_coeffs")

    def step_host(self, u, v, check=True):
        """u, v: host (CPU) float64 contiguous tensors or numpy arrays, updated in place."""
        import numpy as np
        import torch
        ptrs = []
        nb = self.B * self.N
        for a in (u, v):
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == nb
                ptrs.append(ctypes.c_void_p(a.ctypes.data))
            else:
                assert a.device.type == "cpu" and a.dtype == torch.float64 and a.is_contiguous() and a.numel() == nb
                ptrs.append(ctypes.c_void_p(a.data_ptr()))
        infos = self._infos()
        st = _lib().acac_step_host(self.h, ptrs[0], ptrs[1], infos)
        if check:
            _check(st, "acac_step_host")
        return self._out(infos)

    def energy(self, u, v):
        """(energy, mass) of the state; lists of B values for an ensemble."""
        import torch
        e, m = (ctypes.c_double * self.B)(), (ctypes.c_double * self.B)()
        nb = self.B * self.N
        _check(_lib().acac_energy(self.h, _dev(u, torch.float64, nb, "u"), _dev(v, torch.float64, nb, "v"),
                                  e, m), "acac_energy")
        return (e[0], m[0]) if self.B == 1 else (list(e), list(m))

    # -- components
    def residual(self, X1, X0, dt, F):
        import torch
        fn = ctypes.c_double()
        st = _lib().acac_residual(self.h, _dev(X1, torch.float64, 2 * self.N, "X1"),
                                  _dev(X0, torch.float64, 2 * self.N, "X0"), float(dt),
                                  _dev(F, torch.float64, 2 * self.N, "F"), ctypes.byref(fn))
        _check(st, "acac_residual")
        return fn.value

    def jacobian(self, X1, X0, dt, J):
        import torch
        _check(_lib().acac_jacobian(self.h, _dev(X1, torch.float64, 2 * self.N), _dev(X0, torch.float64, 2 * self.N),
                                    float(dt), _dev(J, self.kdtype, 4 * self.nslot * self.N, "J")), "acac_jacobian")

    def spmv(self, J, w, y):
        _check(_lib().acac_spmv(self.h, _dev(J, self.kdtype, 4 * self.nslot * self.N, "J"), _dev(w, self.kdtype, 2 * self.N, "w"),
                                _dev(y, self.kdtype, 2 * self.N, "y")), "acac_spmv")

    def jvp(self, X1, X0, dt, w, y):
        import torch
        _check(_lib().acac_jvp(self.h, _dev(X1, torch.float64, 2 * self.N), _dev(X0, torch.float64, 2 * self.N),
                               float(dt), _dev(w, self.kdtype, 2 * self.N, "w"),
                               _dev(y, self.kdtype, 2 * self.N, "y")), "acac_jvp")

    def ras_factor(self, J):
        _check(_lib().acac_ras_factor(self.h, _dev(J, self.kdtype, 4 * self.nslot * self.N, "J")), "acac_ras_factor")

    def ras_apply(self, r, z):
        _check(_lib().acac_ras_apply(self.h, _dev(r, self.kdtype, 2 * self.N, "r"),
                                     _dev(z, self.kdtype, 2 * self.N, "z")), "acac_ras_apply")

    def gmres(self, X1, X0, dt, b, x, check=True):
        import torch
        its, res = ctypes.c_int(), ctypes.c_double()
        st = _lib().acac_gmres(self.h, _dev(X1, torch.float64, 2 * self.N), _dev(X0, torch.float64, 2 * self.N),
                               float(dt), _dev(b, torch.float64, 2 * self.N, "b"),
                               _dev(x, torch.float64, 2 * self.N, "x"), ctypes.byref(its), ctypes.byref(res))
        if check:
            _check(st, "acac_gmres")
        return its.value, res.value, st

    # -- adjoint (FP64 handles)
    def jacobian_x0(self, X1, X0, dt, J):
        import torch
        _check(_lib().acac_jacobian_x0(self.h, _dev(X1, torch.float64, 2 * self.N), _dev(X0, torch.float64, 2 * self.N),
                                       float(dt), _dev(J, self.kdtype, 4 * self.nslot * self.N, "J")),
               "acac_jacobian_x0")

    def spmv_t(self, J, w, y):
        _check(_lib().acac_spmv_t(self.h, _dev(J, self.kdtype, 4 * self.nslot * self.N, "J"),
                                  _dev(w, self.kdtype, 2 * self.N, "w"), _dev(y, self.kdtype, 2 * self.N, "y")),
               "acac_spmv_t")

    def loss(self, X, target, w_energy, w_misfit, dX):
        """Returns (L, [dL/dalpha, dL/dbeta, dL/dtheta, dL/dgamma]); dX receives dL/dX."""
        import torch
        L, g = ctypes.c_double(), (ctypes.c_double * 4)()
        _check(_lib().acac_loss(self.h, _dev(X, torch.float64, 2 * self.N, "X"),
                                _dev(target, torch.float64, 2 * self.N, "target"), float(w_energy), float(w_misfit),
                                ctypes.byref(L), _dev(dX, torch.float64, 2 * self.N, "dX"), g), "acac_loss")
        return L.value, list(g)

    def adjoint_step(self, X1, X0, dt, lam1, lam0, rtol=1e-10):
        """lam0 = -J0^T mu with J1^T mu = lam1; returns (grad[4], gmres_its)."""
        import torch
        g, its = (ctypes.c_double * 4)(), ctypes.c_int()
        n = 2 * self.N
        _check(_lib().acac_adjoint_step(self.h, _dev(X1, torch.float64, n, "X1"), _dev(X0, torch.float64, n, "X0"),
                                        float(dt), _dev(lam1, torch.float64, n, "lam1"),
                                        _dev(lam0, torch.float64, n, "lam0"), g, float(rtol), ctypes.byref(its)),
               "acac_adjoint_step")
        return list(g), its.value

    def adjoint(self, u0, v0, nsteps, dt, u_target, v_target, w_energy=1.0, w_misfit=1.0, every=5, rtol=1e-10,
                du0=None, dv0=None):
        """Loss of the state after nsteps fixed-dt steps and its gradient.  Returns
        (L, du0, dv0, [dL/dalpha, dL/dbeta, dL/dtheta, dL/dgamma], gmres_its)."""
        import torch
        du0 = torch.empty_like(u0) if du0 is None else du0
        dv0 = torch.empty_like(v0) if dv0 is None else dv0
        L, g, its = ctypes.c_double(), (ctypes.c_double * 4)(), ctypes.c_int()
        _check(_lib().acac_adjoint(self.h, _dev(u0, torch.float64, self.N, "u0"), _dev(v0, torch.float64, self.N, "v0"),
                                   int(nsteps), float(dt), int(every), _dev(u_target, torch.float64, self.N, "u_target"),
                                   _dev(v_target, torch.float64, self.N, "v_target"), float(w_energy), float(w_misfit),
                                   float(rtol), ctypes.byref(L), _dev(du0, torch.float64, self.N, "du0"),
                                   _dev(dv0, torch.float64, self.N, "dv0"), g, ctypes.byref(its)), "acac_adjoint")
        return L.value, du0, dv0, list(g), its.value

    # -- instrumentation
    def profile(self, enable=True, kernels=None):
        """Reset the counters; time every launch (enable), or only the named kernel
        classes (kernels = iterable of names as kernel_stats reports them)."""
        if kernels is None:
            _check(_lib().acac_profile(self.h, 1 if enable else 0), "acac_profile")
            return
        names = [_lib().acac_kernel_name(k).decode() for k in range(NKERNEL)]
        mask = 0
        for k in kernels:
            mask |= 1 << names.index(k)
        _check(_lib().acac_profile_mask(self.h, mask if enable else 0), "acac_profile_mask")

    def kernel_stats(self):
        """{name: (launches, total_ms, algorithmic_bytes, algorithmic_flops)} per kernel class."""
        out = {}
        for k in range(NKERNEL):
            n, ms, b, f = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            _check(_lib().acac_kernel_stats(self.h, k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b),
                                            ctypes.byref(f)), "acac_kernel_stats")
            out[_lib().acac_kernel_name(k).decode()] = (n.value, ms.value, b.value, f.value)
        return out

    def nks_solve(self, U0, dt, U1, check=True):
        import torch
        info = acac_step_info()
        st = _lib().acac_nks_solve(self.h, _dev(U0, torch.float64, 2 * self.N, "U0"), float(dt),
                                   _dev(U1, torch.float64, 2 * self.N, "U1"), ctypes.byref(info))
        if check:
            _check(st, "acac_nks_solve")
        return info
