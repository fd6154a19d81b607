"""GB300 (sm_103a) ReLU-QP solver: Python binding of ``librelu_qp.so``.

This module only marshals arguments to the C ABI declared in
``include/relu_qp.h``; every step of the solve runs in the library's CUDA
kernels.  Importing it does not need a GPU; creating a solver does, and it
fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["ReluQP", "ReluQPError", "lib", "library_path", "OK", "SOLVED", "MAX_ITER", "NUMERICAL",
           "PREC_FP32", "PREC_BF16X3", "PREC_FP64", "PREC_FP64R", "EXPORTED_SYMBOLS", "Info", "Opts", "Prof", "Server", "Result",
           "condense_mpc"]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "librelu_qp.so")

OK = 0
SOLVED, MAX_ITER, NUMERICAL = 0, 1, 2
PREC_FP32, PREC_BF16X3, PREC_FP64, PREC_FP64R = 0, 1, 2, 3
ERRORS = {-1: "INVALID", -2: "NOT_PD", -3: "OOM", -4: "CUDA", -5: "TIMEOUT", -6: "UNSUPPORTED"}

_c_int, _c_double, _c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


class Opts(ctypes.Structure):
    _fields_ = [("check_interval", _c_int), ("adaptive_rho", _c_int), ("rho0", _c_double),
                ("eq_scale", _c_double), ("keep_fp64", _c_int), ("max_batch", _c_int),
                ("batch_precision", _c_int), ("stream", _c_void_p), ("scaling_iters", _c_int),
                ("single_precision", _c_int), ("device_budget", ctypes.c_longlong)]


class Prof(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("layer_launches", ctypes.c_longlong),
                ("layer_timed", ctypes.c_longlong), ("layer_ms", _c_double), ("layer_flops", _c_double),
                ("host_checks", ctypes.c_longlong), ("host_gap_ms", _c_double),
                ("resident_launches", ctypes.c_longlong)]


class Info(ctypes.Structure):
    _fields_ = [("status", _c_int), ("iters", _c_int), ("rho_index", _c_int), ("rho_switches", _c_int),
                ("r_prim", _c_double), ("r_dual", _c_double), ("solve_ms", _c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_longlong), ("family", _c_int), ("client", _c_int), ("status", _c_int),
                ("iters", _c_int), ("rho_index", _c_int), ("rho_switches", _c_int), ("r_prim", _c_double),
                ("r_dual", _c_double), ("t_submit", _c_double), ("t_done", _c_double)]


# name -> (restype, argtypes); the CPU test checks the library exports each one
_SIGNATURES = {
    "relu_qp_default_opts": (None, [ctypes.POINTER(Opts)]),
    "relu_qp_setup": (_c_int, [ctypes.POINTER(_c_void_p), _c_int, _c_int, _dp, _dp, _dp, _dp, _dp, _c_double,
                               _dp, _c_int, ctypes.POINTER(Opts)]),
    "relu_qp_update": (_c_int, [_c_void_p, _dp, _dp, _dp]),
    "relu_qp_solve": (_c_int, [_c_void_p, _dp, _dp, _c_int, _c_double, _c_double, _c_int, _dp, _dp, _dp,
                               ctypes.POINTER(Info)]),
    "relu_qp_solve_noalloc": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_int, _c_double, _c_double, _c_int,
                                       _c_void_p, _c_void_p, _c_void_p, ctypes.POINTER(Info)]),
    "relu_qp_get_layer": (_c_int, [_c_void_p, _c_int, _dp, _dp]),
    "relu_qp_set_opts": (_c_int, [_c_void_p, ctypes.POINTER(Opts)]),
    "relu_qp_dims": (_c_int, [_c_void_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                              ctypes.POINTER(_c_int)]),
    "relu_qp_update_batch": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_void_p, _c_void_p]),
    "relu_qp_set_parametric": (_c_int, [_c_void_p, _c_int, _dp, _dp, _dp, _dp]),
    "relu_qp_update_batch_x0": (_c_int, [_c_void_p, _c_int, _c_void_p]),
    "relu_qp_condense_mpc": (_c_int, [_c_int, _c_int, _c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                      _c_int, _c_void_p, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
    "relu_qp_solve_batch": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_void_p, _c_void_p, _c_double, _c_double, _c_int,
                                     _c_void_p, _c_void_p, _c_void_p, ctypes.POINTER(Info)]),
    "relu_qp_profile": (_c_int, [_c_void_p, _c_int, _c_int, ctypes.POINTER(Prof)]),
    "relu_qp_server_create": (_c_int, [ctypes.POINTER(_c_void_p), ctypes.POINTER(_c_void_p), _c_int,
                                       ctypes.POINTER(_c_int), _c_double, _c_double, _c_int]),
    "relu_qp_server_submit": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p, ctypes.c_longlong]),
    "relu_qp_server_step": (_c_int, [_c_void_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "relu_qp_server_poll": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(Result), _c_void_p, _c_int]),
    "relu_qp_server_clock": (_c_double, [_c_void_p]),
    "relu_qp_server_destroy": (None, [_c_void_p]),
    "relu_qp_server_error": (ctypes.c_char_p, [_c_void_p]),
    "relu_qp_server_set_budget": (_c_int, [_c_void_p, ctypes.c_longlong]),
    "relu_qp_server_family_bytes": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(ctypes.c_longlong)]),
    "relu_qp_server_bytes_in_use": (ctypes.c_longlong, [_c_void_p]),
    "relu_qp_device_bytes": (ctypes.c_longlong, [_c_void_p]),
    "relu_qp_single_config": (_c_int, [_c_void_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                      ctypes.POINTER(_c_int)]),
    "relu_qp_single_set_config": (_c_int, [_c_void_p, _c_int, _c_int]),
    "relu_qp_diag_device_wait": (_c_int, [_c_int, ctypes.c_longlong, ctypes.POINTER(_c_int),
                                          ctypes.POINTER(_c_double)]),
    "relu_qp_diag_host_barrier": (_c_int, [_c_int, _c_int, _c_int, ctypes.c_longlong, ctypes.POINTER(_c_int),
                                           ctypes.POINTER(_c_double)]),
    "relu_qp_destroy": (None, [_c_void_p]),
    "relu_qp_last_error": (ctypes.c_char_p, [_c_void_p]),
}
EXPORTED_SYMBOLS = tuple(_SIGNATURES)

_lib = None


def lib():
    """Load librelu_qp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError(f"{library_path} is missing: build it with "
                               "paper_2311_18056_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(library_path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class ReluQPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"relu_qp error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code
        self.kind = ERRORS.get(code, "?")


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape}, got {a.shape}")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _buf(a, dtype, shape):
    """(pointer, keep-alive) for a host NumPy array or a CUDA torch tensor of the given shape."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        want = torch.float32 if dtype == np.float32 else torch.int32
        if a.dtype != want or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError(f"expected a contiguous {want} tensor of shape {shape}, got {a.dtype} {tuple(a.shape)}")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if arr.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape}, got {arr.shape}")
    return arr.ctypes.data, arr


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


class ReluQP:
    """One QP  min 1/2 x'Px + q'x  s.t.  l <= Ax <= u  with its bank of layers on the GPU.

    Keyword options mirror relu_qp_opts (include/relu_qp.h): check_interval,
    adaptive_rho, rho0, eq_scale, keep_fp64, max_batch (> 0 enables the batched
    entry points), precision (batched: PREC_FP32 or PREC_BF16X3), stream (a CUDA
    stream or its handle), scaling_iters (Algorithm 1's scaling step: modified
    Ruiz iterations at setup, 0 = off), single_precision (single solves:
    PREC_FP32, PREC_FP64 or PREC_FP64R, the FP64-anchored form) and
    device_budget (bytes of device memory the handle may keep, 0 = no cap)."""

    def __init__(self, P, A, l, u, q=None, sigma=1e-6, rho_bank=(0.1, 1.0, 10.0), *, check_interval=25,
                 adaptive_rho=True, rho0=0.1, eq_scale=1e3, keep_fp64=False, max_batch=0,
                 precision=PREC_FP32, stream=None, scaling_iters=0, single_precision=PREC_FP32,
                 device_budget=0):
        L = lib()
        P = _f64(P)
        n = P.shape[0]
        A = _f64(A) if A is not None else np.zeros((0, n))
        m = A.shape[0] if A.ndim == 2 else 0
        l = _f64(l, (m,)) if m else np.zeros(0)
        u = _f64(u, (m,)) if m else np.zeros(0)
        q = _f64(q, (n,))
        bank = _f64(rho_bank)
        o = Opts()
        L.relu_qp_default_opts(ctypes.byref(o))
        o.check_interval = int(check_interval)
        o.adaptive_rho = int(bool(adaptive_rho))
        o.rho0 = float(rho0)
        o.eq_scale = float(eq_scale)
        o.keep_fp64 = int(bool(keep_fp64))
        o.max_batch = int(max_batch)
        o.batch_precision = int(precision)
        o.stream = _stream_handle(stream)
        o.scaling_iters = int(scaling_iters)
        o.single_precision = int(single_precision)
        o.device_budget = int(device_budget)
        h = _c_void_p()
        rc = L.relu_qp_setup(ctypes.byref(h), n, m, _ptr(P), _ptr(q), _ptr(A) if m else None,
                             _ptr(l) if m else None, _ptr(u) if m else None, float(sigma), _ptr(bank),
                             int(bank.size), ctypes.byref(o))
        if rc != OK:
            raise ReluQPError(rc, L.relu_qp_last_error(None).decode())
        self._h = h
        self.n, self.m, self.n_rho = n, m, int(bank.size)
        self.rho_bank = tuple(float(r) for r in bank)

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            raise ReluQPError(rc, lib().relu_qp_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    def device_bytes(self):
        """Device memory the handle keeps (what device_budget caps)."""
        return int(lib().relu_qp_device_bytes(self._h))

    def single_config(self):
        """Launch shape of the single-QP solve: (ctas, cluster, cached_rows); cluster 0 = grid form."""
        c, k, r = _c_int(0), _c_int(0), _c_int(0)
        self._check(lib().relu_qp_single_config(self._h, ctypes.byref(c), ctypes.byref(k), ctypes.byref(r)))
        return c.value, k.value, r.value

    def set_single_config(self, ctas, cluster=0):
        """Use `ctas` CTAs as a grid (cluster 0) or as one cluster (cluster = ctas in 2, 4, 8, 16)."""
        self._check(lib().relu_qp_single_set_config(self._h, int(ctas), int(cluster)))

    def close(self):
        if getattr(self, "_h", None):
            lib().relu_qp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- single QP ----------------------------------------------------------
    def update(self, q=None, l=None, u=None):
        q = _f64(q, (self.n,))
        l = _f64(l, (self.m,))
        u = _f64(u, (self.m,))
        self._check(lib().relu_qp_update(self._h, _ptr(q), _ptr(l), _ptr(u)))

    def solve(self, x_warm=None, lam_warm=None, rho_index=-1, eps_abs=1e-3, eps_rel=0.0, max_iter=4000):
        x_warm = _f64(x_warm, (self.n,))
        lam_warm = _f64(lam_warm, (self.m,))
        x = np.empty(self.n)
        z = np.empty(self.m)
        lam = np.empty(self.m)
        info = Info()
        self._check(lib().relu_qp_solve(self._h, _ptr(x_warm), _ptr(lam_warm), int(rho_index), float(eps_abs),
                                        float(eps_rel), int(max_iter), _ptr(x), _ptr(z) if self.m else None,
                                        _ptr(lam) if self.m else None, ctypes.byref(info)))
        out = info.as_dict()
        out.update(x=x, z=z, lam=lam)
        return out

    # -- batched QPs (same P, A; own q, l, u) -------------------------------
    def update_batch(self, Q, L=None, U=None):
        """Per-QP data: Q (B, n), L and U (B, m), FP32, host arrays or CUDA tensors."""
        B = int(Q.shape[0])
        q, kq = _buf(Q, np.float32, (B, self.n))
        l, kl = _buf(L, np.float32, (B, self.m)) if self.m else (None, None)
        u, ku = _buf(U, np.float32, (B, self.m)) if self.m else (None, None)
        self._check(lib().relu_qp_update_batch(self._h, B, q, l, u))
        self._batch = B

    def set_parametric(self, F, E, l0, u0):
        """q = F x0, l = l0 - E x0, u = u0 - E x0 for the x0-driven batched updates."""
        F = _f64(F)
        nx = F.shape[1]
        E = _f64(E, (self.m, nx)) if self.m else None
        l0 = _f64(l0, (self.m,)) if self.m else None
        u0 = _f64(u0, (self.m,)) if self.m else None
        self._check(lib().relu_qp_set_parametric(self._h, nx, _ptr(F), _ptr(E), _ptr(l0), _ptr(u0)))
        self.nx = nx

    def update_batch_x0(self, X0):
        B = int(X0.shape[0])
        x, kx = _buf(X0, np.float32, (B, self.nx))
        self._check(lib().relu_qp_update_batch_x0(self._h, B, x))
        self._batch = B

    def solve_batch(self, B=None, X_warm=None, Lam_warm=None, rho_warm=None, eps_abs=1e-3, eps_rel=0.0,
                    max_iter=4000, out=None, infos=True):
        """Solve the first B QPs of the last update.  Outputs go to `out` = (X, Z, Lam)
        (CUDA tensors or host arrays) or to new host arrays."""
        B = self._batch if B is None else int(B)
        xw, kxw = _buf(X_warm, np.float32, (B, self.n))
        lw, klw = _buf(Lam_warm, np.float32, (B, self.m)) if self.m else (None, None)
        rw, krw = _buf(rho_warm, np.int32, (B,))
        if out is None:
            out = (np.empty((B, self.n), np.float32), np.empty((B, self.m), np.float32),
                   np.empty((B, self.m), np.float32))
        xo, kxo = _buf(out[0], np.float32, (B, self.n))
        zo, kzo = _buf(out[1], np.float32, (B, self.m)) if self.m and out[1] is not None else (None, None)
        lo, klo = _buf(out[2], np.float32, (B, self.m)) if self.m and out[2] is not None else (None, None)
        inf = (Info * B)() if infos else None
        self._check(lib().relu_qp_solve_batch(self._h, B, xw, lw, rw, float(eps_abs), float(eps_rel), int(max_iter),
                                              xo, zo, lo, inf))
        res = {"x": out[0], "z": out[1], "lam": out[2]}
        if infos:
            res["status"] = np.array([i.status for i in inf])
            res["iters"] = np.array([i.iters for i in inf])
            res["rho_index"] = np.array([i.rho_index for i in inf])
            res["rho_switches"] = np.array([i.rho_switches for i in inf])
            res["r_prim"] = np.array([i.r_prim for i in inf])
            res["r_dual"] = np.array([i.r_dual for i in inf])
            res["solve_ms"] = inf[0].solve_ms if B else 0.0
        return res

    def profile(self, enable=-1, reset=False):
        """Counters of relu_qp_profile as a dict; enable: 1 on, 0 off, -1 unchanged."""
        pr = Prof()
        self._check(lib().relu_qp_profile(self._h, int(enable), int(bool(reset)), ctypes.byref(pr)))
        return {k: getattr(pr, k) for k, _ in pr._fields_}

    def get_layer(self, rho_index):
        R = self.n + self.m
        Wt = np.empty((R, R))
        Bop = np.empty((R, self.n))
        self._check(lib().relu_qp_get_layer(self._h, int(rho_index), _ptr(Wt), _ptr(Bop)))
        return Wt, Bop

    def set_opts(self, check_interval=None, adaptive_rho=None, rho0=None):
        o = Opts()
        lib().relu_qp_default_opts(ctypes.byref(o))
        o.check_interval = 25 if check_interval is None else int(check_interval)
        o.adaptive_rho = 1 if adaptive_rho is None else int(bool(adaptive_rho))
        o.rho0 = 0.1 if rho0 is None else float(rho0)
        self._check(lib().relu_qp_set_opts(self._h, ctypes.byref(o)))


def condense_mpc(A, B, Q, R, N, QN=None, umin=None, umax=None, xmin=None, xmax=None, K=None,
                 lqr_precondition=True, stream=None):
    """LQR-preconditioned condensing of the MPC problem x+ = A x + B u (Sec. IV) on the GPU in FP64.

    Returns dict(P, A, F, E, l0, u0, K): the QP min 1/2 du'P du + (F x0)'du,
    l0 - E x0 <= A du <= u0 - E x0 over du = [du_0; ..; du_{N-1}], the rows being
    the control limits of every stage, then (with xmin/xmax) the state limits."""
    L = lib()
    A = _f64(A)
    B = _f64(B)
    nx, nu, N = A.shape[0], B.shape[1], int(N)
    Q = _f64(Q, (nx, nx))
    R = _f64(R, (nu, nu))
    QN = _f64(QN, (nx, nx))
    umin, umax = _f64(umin, (nu,)), _f64(umax, (nu,))
    xmin, xmax = _f64(xmin, (nx,)), _f64(xmax, (nx,))
    K = _f64(K, (nu, nx))
    n = N * nu
    m = N * nu + (N * nx if (xmin is not None or xmax is not None) else 0)
    P, Acon, F, E = np.empty((n, n)), np.empty((m, n)), np.empty((n, nx)), np.empty((m, nx))
    l0, u0, Kout = np.empty(m), np.empty(m), np.empty((nu, nx))
    rc = L.relu_qp_condense_mpc(nx, nu, N, _ptr(A), _ptr(B), _ptr(Q), _ptr(R), _ptr(QN), _ptr(umin), _ptr(umax),
                                _ptr(xmin), _ptr(xmax), _ptr(K), int(bool(lqr_precondition)),
                                _stream_handle(stream), _ptr(P), _ptr(Acon), _ptr(F), _ptr(E), _ptr(l0), _ptr(u0),
                                _ptr(Kout))
    if rc != OK:
        raise ReluQPError(rc, L.relu_qp_last_error(None).decode())
    return {"P": P, "A": Acon, "F": F, "E": E, "l0": l0, "u0": u0, "K": Kout}


class Server:
    """Continuous batching of MPC requests over several resident problem families.

    ``families`` are ReluQP handles set up with max_batch > 0 and
    set_parametric(); a request is a new initial state x0 for one client of one
    family.  See relu_qp_server_* in include/relu_qp.h.
    """

    def __init__(self, families, clients=None, eps_abs=1e-3, eps_rel=0.0, max_iter=4000):
        L = lib()
        self.families = list(families)
        nf = len(self.families)
        hs = (_c_void_p * nf)(*[f.handle for f in self.families])
        cl = (_c_int * nf)(*([0] * nf if clients is None else [int(c) for c in clients]))
        s = _c_void_p()
        rc = L.relu_qp_server_create(ctypes.byref(s), hs, nf, cl, float(eps_abs), float(eps_rel), int(max_iter))
        if rc != OK:
            raise ReluQPError(rc, L.relu_qp_last_error(None).decode())
        self._s = s
        self._nmax = max(f.n for f in self.families)

    def submit(self, family, x0, client=-1, tag=0):
        x = np.ascontiguousarray(np.asarray(x0, dtype=np.float32))
        if x.size != self.families[family].nx:
            raise ValueError("x0 must have nx entries")
        rc = lib().relu_qp_server_submit(self._s, int(family), int(client), x.ctypes.data, int(tag))
        if rc != OK:
            raise ReluQPError(rc, "invalid request (family, client or non-finite x0)")

    def step(self):
        a, w = _c_int(), _c_int()
        rc = lib().relu_qp_server_step(self._s, ctypes.byref(a), ctypes.byref(w))
        if rc != OK:
            raise ReluQPError(rc, lib().relu_qp_server_error(self._s).decode())
        return a.value, w.value

    def poll(self, max_results=4096):
        res = (Result * max_results)()
        x = np.empty((max_results, self._nmax), np.float32)
        k = lib().relu_qp_server_poll(self._s, max_results, res, x.ctypes.data, self._nmax)
        out = []
        for i in range(k):
            r = {f: getattr(res[i], f) for f, _ in Result._fields_}
            r["x"] = x[i, :self.families[r["family"]].n].copy()
            out.append(r)
        return out

    def clock(self):
        return lib().relu_qp_server_clock(self._s)

    def set_budget(self, nbytes):
        """Device-memory budget for admission (bytes; 0 = free slots only)."""
        rc = lib().relu_qp_server_set_budget(self._s, int(nbytes))
        if rc != OK:
            raise ReluQPError(rc, lib().relu_qp_server_error(self._s).decode())

    def family_bytes(self, family):
        """(fixed bytes, bytes per admitted request) of one family."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        rc = lib().relu_qp_server_family_bytes(self._s, int(family), ctypes.byref(a), ctypes.byref(b))
        if rc != OK:
            raise ReluQPError(rc, "family out of range")
        return a.value, b.value

    def bytes_in_use(self):
        """Bytes charged by the requests now in slots."""
        return int(lib().relu_qp_server_bytes_in_use(self._s))

    def close(self):
        if getattr(self, "_s", None):
            lib().relu_qp_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
