"""Thin Python binding of ``libipm.so`` (the C ABI of ``include/ipm.h``).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  Device buffers and streams come from PyTorch (``tensor.data_ptr()``
and ``torch.cuda.current_stream().cuda_stream``).  There is no CPU fallback:
if the library is missing or cannot load, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libipm.so")

IPM_OK = 0
STATUS = {0: "IPM_OK", 1: "IPM_ERR_ARG", 2: "IPM_ERR_CUDA", 3: "IPM_ERR_OOM",
          4: "IPM_ERR_SINGULAR_GX", 5: "IPM_ERR_NOT_PD", 6: "IPM_ERR_LINESEARCH",
          7: "IPM_ERR_MAXITER", 8: "IPM_ERR_TIMEOUT", 9: "IPM_ERR_STATE"}
PREC_FP64, PREC_MIXED = 0, 1
Q_KHAT, Q_RHS_U, Q_Z, Q_FGH, Q_JAC, Q_HESS, Q_ERRS, Q_INFO, Q_TIMERS = range(9)
N_PHASES = 9
PHASES = ("eval", "condense_K", "lu", "zsolve", "gemm", "reduced_rhs", "cholesky", "recover", "linesearch")


class IPMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.kind = STATUS.get(status, str(status))


_I = ctypes.POINTER(ctypes.c_int)
_D = ctypes.POINTER(ctypes.c_double)


class Network(ctypes.Structure):
    _fields_ = [("n_bus", ctypes.c_int), ("n_line", ctypes.c_int), ("n_gen", ctypes.c_int),
                ("from_", _I), ("to", _I), ("gen_bus", _I),
                ("r", _D), ("x", _D), ("b", _D), ("pmax", _D), ("qmax", _D),
                ("c2", _D), ("c1", _D), ("vmin", _D), ("vmax", _D)]


BARRIER_MONOTONE, BARRIER_ADAPTIVE = 0, 1


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("panel", ctypes.c_int), ("barrier_rule", ctypes.c_int),
                ("reserved", ctypes.c_int * 6), ("sigma", ctypes.c_double)]


class Dims(ctypes.Structure):
    _fields_ = [("n_bus", ctypes.c_int), ("n_line", ctypes.c_int), ("n_gen", ctypes.c_int),
                ("n_scen", ctypes.c_int), ("n_x", ctypes.c_int), ("n_u", ctypes.c_int), ("m", ctypes.c_int),
                ("state_len", ctypes.c_longlong), ("step_len", ctypes.c_longlong),
                ("nnz_lu", ctypes.c_longlong), ("lu_levels", ctypes.c_int)]


_lib = None


def load():
    """Load libipm.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2301_04869_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, c_int, c_double, c_ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "ipm_default_options": (c_int, [ctypes.POINTER(Options)]),
        "ipm_create": (c_int, [ctypes.POINTER(Network), c_int, _D, _D, ctypes.POINTER(Options), ctypes.POINTER(vp)]),
        "ipm_destroy": (c_int, [vp]),
        "ipm_get_dims": (c_int, [vp, ctypes.POINTER(Dims)]),
        "ipm_last_error": (ctypes.c_char_p, [vp]),
        "ipm_init_state": (c_int, [vp, vp]),
        "ipm_set_state": (c_int, [vp, vp, c_int, vp]),
        "ipm_get_state": (c_int, [vp, vp, c_int, vp]),
        "ipm_eval_derivatives": (c_int, [vp, vp]),
        "ipm_condense_scenarios": (c_int, [vp, vp]),
        "ipm_factor_schur": (c_int, [vp, c_double, _I, vp]),
        "ipm_solve_kkt": (c_int, [vp, vp, _D, vp]),
        "ipm_step": (c_int, [vp, _I, _D, vp]),
        "ipm_solve": (c_int, [vp, _I, _D, vp]),
        "ipm_get_quantity": (c_int, [vp, c_int, c_int, _D, c_ll, vp]),
        "ipm_set_profiling": (c_int, [vp, c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Solver:
    """One context: a network with N load scenarios on the current GPU."""

    def __init__(self, net, pd, qd, precision=PREC_FP64, tol=1e-8, max_iter=200, max_refine=25,
                 barrier_rule=None, sigma=None):
        lib = load()
        self._lib = lib
        self._keep = dict(
            fr=np.ascontiguousarray(net.fr, dtype=np.int32), to=np.ascontiguousarray(net.to, dtype=np.int32),
            gen=np.ascontiguousarray(net.gen_bus, dtype=np.int32),
            r=np.ascontiguousarray(net.r, dtype=np.float64), x=np.ascontiguousarray(net.x, dtype=np.float64),
            b=np.ascontiguousarray(net.b, dtype=np.float64),
            pmax=np.ascontiguousarray(net.pmax, dtype=np.float64), qmax=np.ascontiguousarray(net.qmax, dtype=np.float64),
            c2=np.ascontiguousarray(net.c2, dtype=np.float64), c1=np.ascontiguousarray(net.c1, dtype=np.float64),
            vmin=np.ascontiguousarray(net.vmin, dtype=np.float64), vmax=np.ascontiguousarray(net.vmax, dtype=np.float64))
        k = self._keep
        cnet = Network(int(net.n_bus), int(k["fr"].size), int(k["gen"].size),
                       _ptr(k["fr"], ctypes.c_int), _ptr(k["to"], ctypes.c_int), _ptr(k["gen"], ctypes.c_int),
                       _ptr(k["r"], ctypes.c_double), _ptr(k["x"], ctypes.c_double), _ptr(k["b"], ctypes.c_double),
                       _ptr(k["pmax"], ctypes.c_double), _ptr(k["qmax"], ctypes.c_double),
                       _ptr(k["c2"], ctypes.c_double), _ptr(k["c1"], ctypes.c_double),
                       _ptr(k["vmin"], ctypes.c_double), _ptr(k["vmax"], ctypes.c_double))
        opt = Options()
        lib.ipm_default_options(ctypes.byref(opt))
        opt.tol = tol
        opt.max_iter = max_iter
        opt.precision = precision
        opt.max_refine = max_refine
        if barrier_rule is not None:
            opt.barrier_rule = barrier_rule
        if sigma is not None:
            opt.sigma = sigma
        pd = np.ascontiguousarray(np.atleast_2d(pd), dtype=np.float64)
        qd = np.ascontiguousarray(np.atleast_2d(qd), dtype=np.float64)
        self.N = pd.shape[0]
        h = ctypes.c_void_p()
        st = lib.ipm_create(ctypes.byref(cnet), self.N, _ptr(pd, ctypes.c_double), _ptr(qd, ctypes.c_double),
                            ctypes.byref(opt), ctypes.byref(h))
        if st != IPM_OK:
            raise IPMError(st, "ipm_create failed")
        self._h = h
        d = Dims()
        lib.ipm_get_dims(h, ctypes.byref(d))
        self.dims = d

    # -- plumbing ---------------------------------------------------------
    def _check(self, st):
        if st != IPM_OK:
            raise IPMError(st, self._lib.ipm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ipm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI, same names --------------------------------------------------
    def ipm_init_state(self, stream=None):
        self._check(self._lib.ipm_init_state(self._h, _stream(stream)))

    def ipm_set_state(self, state, stream=None):
        """state: CUDA tensor (float64, state_len) or numpy array (host)."""
        if isinstance(state, np.ndarray):
            a = np.ascontiguousarray(state, dtype=np.float64)
            assert a.size == self.dims.state_len
            self._check(self._lib.ipm_set_state(self._h, a.ctypes.data_as(ctypes.c_void_p), 0, _stream(stream)))
        else:
            assert state.is_cuda and state.dtype.is_floating_point and state.numel() == self.dims.state_len
            self._check(self._lib.ipm_set_state(self._h, ctypes.c_void_p(state.data_ptr()), 1, _stream(stream)))

    def ipm_get_state(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.dims.state_len)
        if isinstance(out, np.ndarray):
            self._check(self._lib.ipm_get_state(self._h, out.ctypes.data_as(ctypes.c_void_p), 0, _stream(stream)))
        else:
            self._check(self._lib.ipm_get_state(self._h, ctypes.c_void_p(out.data_ptr()), 1, _stream(stream)))
        return out

    def ipm_eval_derivatives(self, stream=None):
        self._check(self._lib.ipm_eval_derivatives(self._h, _stream(stream)))

    def ipm_condense_scenarios(self, stream=None):
        self._check(self._lib.ipm_condense_scenarios(self._h, _stream(stream)))

    def ipm_factor_schur(self, delta_w=0.0, stream=None):
        pd = ctypes.c_int(0)
        self._check(self._lib.ipm_factor_schur(self._h, float(delta_w), ctypes.byref(pd), _stream(stream)))
        return bool(pd.value)

    def ipm_solve_kkt(self, step=None, stream=None):
        rr = ctypes.c_double(0.0)
        ptr = ctypes.c_void_p(step.data_ptr()) if step is not None else None
        self._check(self._lib.ipm_solve_kkt(self._h, ptr, ctypes.byref(rr), _stream(stream)))
        return rr.value

    def ipm_step(self, stream=None):
        conv = ctypes.c_int(0)
        err = ctypes.c_double(0.0)
        self._check(self._lib.ipm_step(self._h, ctypes.byref(conv), ctypes.byref(err), _stream(stream)))
        return bool(conv.value), err.value

    def ipm_solve(self, stream=None):
        it = ctypes.c_int(0)
        err = ctypes.c_double(0.0)
        self._check(self._lib.ipm_solve(self._h, ctypes.byref(it), ctypes.byref(err), _stream(stream)))
        return it.value, err.value

    def ipm_get_quantity(self, which, scen=0, stream=None):
        d = self.dims
        sizes = {Q_KHAT: d.n_u * d.n_u, Q_RHS_U: d.n_u, Q_Z: d.n_x * d.n_u, Q_FGH: 1 + d.n_x + d.m,
                 Q_JAC: d.n_x * d.n_x + d.n_x * d.n_u + d.m * d.n_x + d.m * d.n_u,
                 Q_HESS: d.n_x * d.n_x + d.n_x * d.n_u + d.n_u * d.n_u, Q_ERRS: 6, Q_INFO: 10,
                 Q_TIMERS: 2 * N_PHASES + 1}
        out = np.empty(sizes[which])
        self._check(self._lib.ipm_get_quantity(self._h, which, scen, _ptr(out, ctypes.c_double), out.size,
                                               _stream(stream)))
        return out

    def ipm_set_profiling(self, on=1):
        self._check(self._lib.ipm_set_profiling(self._h, int(on)))

    def timers(self):
        """dict phase -> (ms, calls), plus the library's total kernel launches."""
        t = self.ipm_get_quantity(Q_TIMERS)
        return {p: (t[i], t[N_PHASES + i]) for i, p in enumerate(PHASES)}, int(t[2 * N_PHASES])

    # -- state layout helpers -----------------------------------------------
    def split_state(self, v):
        """Views of a state vector: dict of blocks (see include/ipm.h)."""
        d = self.dims
        N, nx, nu, m = d.n_scen, d.n_x, d.n_u, d.m
        out, o = {}, 0
        for name, shape in [("x", (N, nx)), ("u", (nu,)), ("s", (N, m)), ("y", (N, nx)), ("z", (N, m)),
                            ("zl_x", (N, nx)), ("zu_x", (N, nx)), ("zl_u", (nu,)), ("zu_u", (nu,)),
                            ("zl_s", (N, m)), ("zu_s", (N, m))]:
            k = int(np.prod(shape))
            out[name] = v[o:o + k].reshape(shape)
            o += k
        out["mu"], out["rho"], out["delta_last"] = v[o], v[o + 1], v[o + 2]
        return out

    def pack_state(self, st):
        """Inverse of split_state for a dict with the same keys (e.g. the oracle's)."""
        parts = [np.asarray(st[k], dtype=np.float64).ravel() for k in
                 ("x", "u", "s", "y", "z", "zl_x", "zu_x", "zl_u", "zu_u", "zl_s", "zu_s")]
        parts.append(np.array([st["mu"], st["rho"], st["delta_last"]], dtype=np.float64))
        v = np.concatenate(parts)
        assert v.size == self.dims.state_len
        return v

    def split_step(self, v):
        d = self.dims
        N, nx, nu, m = d.n_scen, d.n_x, d.n_u, d.m
        o = 0
        out = {}
        for name, shape in [("px", (N, nx)), ("pu", (nu,)), ("ps", (N, m)), ("py", (N, nx)), ("pz", (N, m))]:
            k = int(np.prod(shape))
            out[name] = v[o:o + k].reshape(shape)
            o += k
        return out
