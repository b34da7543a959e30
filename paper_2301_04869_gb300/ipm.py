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
PREC_FP64, PREC_MIXED, PREC_FP64_TC = 0, 1, 2
Q_KHAT, Q_RHS_U, Q_Z, Q_FGH, Q_JAC, Q_HESS, Q_ERRS, Q_INFO, Q_TIMERS, Q_ZTZ = range(10)
N_PHASES = 12
PHASES = ("eval", "condense_K", "lu", "zsolve", "gemm", "reduced_rhs", "cholesky", "recover", "linesearch", "split",
          "fallback", "solve1")


class IPMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.kind = STATUS.get(status, str(status))


_I = ctypes.POINTER(ctypes.c_int)
_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)


class Network(ctypes.Structure):
    _fields_ = [("n_bus", ctypes.c_int), ("n_line", ctypes.c_int), ("n_gen", ctypes.c_int),
                ("from_", _I), ("to", _I), ("gen_bus", _I),
                ("r", _D), ("x", _D), ("b", _D), ("pmax", _D), ("qmax", _D),
                ("c2", _D), ("c1", _D), ("vmin", _D), ("vmax", _D), ("rate", _D)]


BARRIER_MONOTONE, BARRIER_ADAPTIVE = 0, 1
REDUCTION_DENSE, REDUCTION_ADJOINT, REDUCTION_AUTO = 0, 1, 2


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("solve_threads", ctypes.c_int), ("barrier_rule", ctypes.c_int),
                ("graphs", ctypes.c_int), ("autotune", ctypes.c_int), ("poison", ctypes.c_int),
                ("lu_pair", ctypes.c_int), ("aug_refine", ctypes.c_int), ("reduction", ctypes.c_int), ("big_block", ctypes.c_int),
                ("sigma", ctypes.c_double), ("tc_solve", ctypes.c_int)]


class Dims(ctypes.Structure):
    _fields_ = [("n_bus", ctypes.c_int), ("n_line", ctypes.c_int), ("n_gen", ctypes.c_int),
                ("n_scen", ctypes.c_int), ("n_x", ctypes.c_int), ("n_u", ctypes.c_int), ("m", ctypes.c_int),
                ("state_len", ctypes.c_longlong), ("step_len", ctypes.c_longlong),
                ("nnz_lu", ctypes.c_longlong), ("lu_levels", ctypes.c_int),
                ("nnz_kx", ctypes.c_int), ("nnz_ku", ctypes.c_int), ("nd", ctypes.c_int),
                ("big_block", ctypes.c_int), ("lu_sparse_ops", ctypes.c_longlong)]


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
        "ipm_set_loads": (c_int, [vp, _D, _D, vp]),
        "ipm_set_contingencies": (c_int, [vp, _I, vp]),
        "ipm_mlp_create": (c_int, [c_int, c_int, c_int, c_int, ctypes.c_ulonglong, ctypes.POINTER(vp)]),
        "ipm_mlp_destroy": (c_int, [vp]),
        "ipm_mlp_param_count": (c_ll, [vp]),
        "ipm_mlp_set_params": (c_int, [vp, _F]),
        "ipm_mlp_get_params": (c_int, [vp, _F]),
        "ipm_mlp_set_normalization": (c_int, [vp, _F, _F, _F, _F]),
        "ipm_mlp_forward": (c_int, [vp, vp, c_int, vp, vp]),
        "ipm_mlp_gradients": (c_int, [vp, vp, vp, c_int, _F, _F, vp]),
        "ipm_mlp_train_step": (c_int, [vp, vp, vp, c_int, ctypes.c_float, _F, vp]),
        "ipm_schur_sum_tc": (c_int, [vp, vp, c_int, c_int, c_int, vp, vp]),
        "ipm_schur_sum_noalloc": (c_int, [vp, vp, vp, vp, c_int, c_int, c_int, vp, vp]),
        "ipm_warm_dim": (c_int, [vp, _I]),
        "ipm_warm_target": (c_int, [vp, vp, vp]),
        "ipm_warm_start": (c_int, [vp, vp, vp]),
        "ipm_kernel_launches": (c_ll, []),
        "ipm_selftest_bounded_wait": (c_int, [c_ll, vp]),
        "ipm_symbolic_export": (c_int, [ctypes.POINTER(Network), c_int, ctypes.POINTER(ctypes.c_int), c_ll,
                                        ctypes.POINTER(c_ll)]),
        "ipm_batch_default_options": (c_int, [ctypes.POINTER(BatchOptions)]),
        "ipm_solve_batch": (c_int, [ctypes.POINTER(vp), c_int, ctypes.POINTER(vp), ctypes.POINTER(BatchOptions),
                                    _I, _D, _I, _D]),
        "ipm_run_instances": (c_int, [ctypes.POINTER(Network), c_int, _I, ctypes.POINTER(_D), ctypes.POINTER(_D),
                                      ctypes.POINTER(Options), ctypes.POINTER(BatchOptions), c_ll,
                                      ctypes.POINTER(_D), _I, _D, _I, _D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def selftest_bounded_wait(polls, stream=None):
    """Status of ipm_selftest_bounded_wait (IPM_ERR_TIMEOUT expected)."""
    return int(load().ipm_selftest_bounded_wait(int(polls), _stream(stream)))


def kernel_launches():
    """Kernels libipm.so has launched in this process (all contexts)."""
    return int(load().ipm_kernel_launches())


SYM_NAMES = ["dims", "lu_colptr", "lu_row", "fr_ptr", "fr_col", "fr_lslot", "gu_ptr", "gu_col", "zp_lev_off",
             "zp_lev_ptr", "zp_rows", "zp_eptr", "zp_col", "zp_slot", "zp_zptr", "zp_zrows", "zp_tptr", "zp_tcol",
             "zp_tslot", "tw_len", "tw_l", "tw_u", "tw_e", "lu_slot"]
SYM_FORCE_BIG = 0x100


def symbolic_export(net, name, force_big=False):
    """One integer structure of the host-side symbolic analysis of `net`
    (ipm_symbolic_export; no GPU needed) as an int32 array; force_big builds
    the structures of the large-trailing-block mode."""
    lib = load()
    keep, cnet = _cnet(net)
    which = SYM_NAMES.index(name) | (SYM_FORCE_BIG if force_big else 0)
    n = ctypes.c_longlong(0)
    st = lib.ipm_symbolic_export(ctypes.byref(cnet), which, None, 0, ctypes.byref(n))
    if st != IPM_OK:
        raise IPMError(st, "ipm_symbolic_export failed")
    out = np.empty(n.value, dtype=np.int32)
    st = lib.ipm_symbolic_export(ctypes.byref(cnet), which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 out.size, ctypes.byref(n))
    if st != IPM_OK:
        raise IPMError(st, "ipm_symbolic_export failed")
    del keep
    return out


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _cnet(net):
    """ipm_network view of a synth.Network (the arrays it points to are returned too)."""
    keep = dict(
        fr=np.ascontiguousarray(net.fr, dtype=np.int32), to=np.ascontiguousarray(net.to, dtype=np.int32),
        gen=np.ascontiguousarray(net.gen_bus, dtype=np.int32),
        r=np.ascontiguousarray(net.r, dtype=np.float64), x=np.ascontiguousarray(net.x, dtype=np.float64),
        b=np.ascontiguousarray(net.b, dtype=np.float64),
        pmax=np.ascontiguousarray(net.pmax, dtype=np.float64), qmax=np.ascontiguousarray(net.qmax, dtype=np.float64),
        c2=np.ascontiguousarray(net.c2, dtype=np.float64), c1=np.ascontiguousarray(net.c1, dtype=np.float64),
        vmin=np.ascontiguousarray(net.vmin, dtype=np.float64), vmax=np.ascontiguousarray(net.vmax, dtype=np.float64))
    rate = getattr(net, "rate", None)
    if rate is not None:
        keep["rate"] = np.ascontiguousarray(rate, dtype=np.float64)
    k = keep
    cnet = Network(int(net.n_bus), int(k["fr"].size), int(k["gen"].size),
                   _ptr(k["fr"], ctypes.c_int), _ptr(k["to"], ctypes.c_int), _ptr(k["gen"], ctypes.c_int),
                   _ptr(k["r"], ctypes.c_double), _ptr(k["x"], ctypes.c_double), _ptr(k["b"], ctypes.c_double),
                   _ptr(k["pmax"], ctypes.c_double), _ptr(k["qmax"], ctypes.c_double),
                   _ptr(k["c2"], ctypes.c_double), _ptr(k["c1"], ctypes.c_double),
                   _ptr(k["vmin"], ctypes.c_double), _ptr(k["vmax"], ctypes.c_double),
                   _ptr(k["rate"], ctypes.c_double) if "rate" in k else None)
    return keep, cnet


def make_options(precision=PREC_FP64, tol=1e-8, max_iter=200, max_refine=60, barrier_rule=None, sigma=None,
                 graphs=False, autotune=False, solve_threads=0, poison=False, lu_pair=True, aug_refine=None,
                 reduction=None, big_block=False, tc_solve=True):
    lib = load()
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
    opt.graphs = int(bool(graphs))
    opt.autotune = int(bool(autotune))
    opt.solve_threads = int(solve_threads)
    opt.poison = int(bool(poison))
    opt.lu_pair = int(bool(lu_pair))
    if aug_refine is not None:
        opt.aug_refine = int(aug_refine)
    if reduction is not None:
        opt.reduction = int(reduction)
    opt.big_block = int(bool(big_block))
    opt.tc_solve = int(bool(tc_solve))
    return opt


class Solver:
    """One context: a network with N load scenarios on the current GPU."""

    def __init__(self, net, pd, qd, precision=PREC_FP64, tol=1e-8, max_iter=200, max_refine=60,
                 barrier_rule=None, sigma=None, graphs=False, autotune=False, solve_threads=0, poison=False,
                 lu_pair=True, aug_refine=None, reduction=None, big_block=False, tc_solve=True):
        lib = load()
        self._lib = lib
        self._keep, cnet = _cnet(net)
        opt = make_options(precision=precision, tol=tol, max_iter=max_iter, max_refine=max_refine,
                           barrier_rule=barrier_rule, sigma=sigma, graphs=graphs, autotune=autotune,
                           solve_threads=solve_threads, poison=poison, lu_pair=lu_pair,
                           aug_refine=aug_refine, reduction=reduction, big_block=big_block,
                           tc_solve=tc_solve)
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

    def ipm_set_loads(self, pd, qd, stream=None):
        pd = np.ascontiguousarray(np.atleast_2d(pd), dtype=np.float64)
        qd = np.ascontiguousarray(np.atleast_2d(qd), dtype=np.float64)
        assert pd.shape == (self.N, self.dims.n_bus) and qd.shape == pd.shape
        self._check(self._lib.ipm_set_loads(self._h, _ptr(pd, ctypes.c_double), _ptr(qd, ctypes.c_double),
                                            _stream(stream)))

    def ipm_set_contingencies(self, trip, stream=None):
        """trip: int per scenario (line out of service, -1 none) or None."""
        if trip is None:
            self._check(self._lib.ipm_set_contingencies(self._h, None, _stream(stream)))
            return
        t = np.ascontiguousarray(trip, dtype=np.int32)
        assert t.shape == (self.N,)
        self._check(self._lib.ipm_set_contingencies(self._h, _ptr(t, ctypes.c_int), _stream(stream)))

    def ipm_get_quantity(self, which, scen=0, stream=None):
        d = self.dims
        sizes = {Q_KHAT: d.n_u * d.n_u, Q_RHS_U: d.n_u, Q_Z: d.n_x * d.n_u, Q_FGH: 1 + d.n_x + d.m,
                 Q_JAC: d.n_x * d.n_x + d.n_x * d.n_u + d.m * d.n_x + d.m * d.n_u,
                 Q_HESS: d.n_x * d.n_x + d.n_x * d.n_u + d.n_u * d.n_u, Q_ERRS: 6, Q_INFO: 19,
                 Q_TIMERS: 2 * N_PHASES + 1, Q_ZTZ: d.n_u * d.n_u}
        out = np.empty(sizes[which])
        self._check(self._lib.ipm_get_quantity(self._h, which, scen, _ptr(out, ctypes.c_double), out.size,
                                               _stream(stream)))
        return out

    def ipm_warm_dim(self):
        d = ctypes.c_int(0)
        self._check(self._lib.ipm_warm_dim(self._h, ctypes.byref(d)))
        return d.value

    def ipm_warm_target(self, out, stream=None):
        """Warm-start vectors of the current state into a device FP32 tensor [N][d]."""
        self._check(self._lib.ipm_warm_target(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def ipm_warm_start(self, pred, stream=None):
        """Start from predicted warm-start vectors (device FP32 tensor [N][d])."""
        self._check(self._lib.ipm_warm_start(self._h, ctypes.c_void_p(pred.data_ptr()), _stream(stream)))

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


class BatchOptions(ctypes.Structure):
    _fields_ = [("n_threads", ctypes.c_int), ("group_contraction", ctypes.c_int), ("window_us", ctypes.c_double),
                ("reserved", ctypes.c_int * 4)]


BATCH_N_STATS = 8
BATCH_STATS = ("grouped_launches", "work_items", "instances_per_launch", "max_active", "wall_ms")


def batch_options(n_threads=8, group_contraction=True, window_us=2000.0):
    lib = load()
    o = BatchOptions()
    lib.ipm_batch_default_options(ctypes.byref(o))
    o.n_threads = int(n_threads)
    o.group_contraction = int(bool(group_contraction))
    o.window_us = float(window_us)
    return o


def ipm_solve_batch(solvers, streams=None, n_threads=8, group_contraction=True, window_us=2000.0):
    """Solve existing contexts together (ipm_solve_batch).  streams: None (the
    runner makes its own) or one torch stream per solver.  Returns
    (iters, kkt_err, status, stats) with stats a dict of BATCH_STATS."""
    lib = load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s._h.value for s in solvers])
    sp = None if streams is None else (ctypes.c_void_p * n)(*[s.cuda_stream for s in streams])
    it = np.zeros(n, dtype=np.int32)
    er = np.zeros(n)
    stt = np.zeros(n, dtype=np.int32)
    stats = np.zeros(BATCH_N_STATS)
    bo = batch_options(n_threads, group_contraction, window_us)
    lib.ipm_solve_batch(hs, n, sp, ctypes.byref(bo), _ptr(it, ctypes.c_int), _ptr(er, ctypes.c_double),
                        _ptr(stt, ctypes.c_int), _ptr(stats, ctypes.c_double))
    return it, er, stt, dict(zip(BATCH_STATS, stats[:len(BATCH_STATS)]))


def ipm_run_instances(nets, pds, qds, mem_budget, precision=PREC_FP64, tol=1e-8, max_iter=200, n_threads=8,
                      group_contraction=True, window_us=2000.0, want_states=False, **opt_kw):
    """Create, solve and destroy independent instances under a device memory
    budget in bytes (ipm_run_instances).  pds[i], qds[i]: [N_i][n_bus_i].
    Returns (iters, kkt_err, status, stats, states) with states a list of
    final state vectors (or None)."""
    lib = load()
    n = len(nets)
    keeps = [_cnet(net) for net in nets]
    arr = (Network * n)(*[k[1] for k in keeps])
    pdl = [np.ascontiguousarray(np.atleast_2d(p), dtype=np.float64) for p in pds]
    qdl = [np.ascontiguousarray(np.atleast_2d(q), dtype=np.float64) for q in qds]
    ns = np.array([p.shape[0] for p in pdl], dtype=np.int32)
    pp = (_D * n)(*[_ptr(p, ctypes.c_double) for p in pdl])
    qp = (_D * n)(*[_ptr(q, ctypes.c_double) for q in qdl])
    states = None
    sp = None
    if want_states:
        states = []
        for net, N in zip(nets, ns):
            nb, ng = int(net.n_bus), int(len(net.gen_bus))
            nx, nu, m = (nb - 1) + (nb - ng), 2 * ng - 1, ng + 1
            states.append(np.zeros(4 * N * nx + 4 * N * m + 3 * nu + 3))
        sp = (_D * n)(*[_ptr(v, ctypes.c_double) for v in states])
    opt = make_options(precision=precision, tol=tol, max_iter=max_iter, **opt_kw)
    bo = batch_options(n_threads, group_contraction, window_us)
    it = np.zeros(n, dtype=np.int32)
    er = np.zeros(n)
    stt = np.zeros(n, dtype=np.int32)
    stats = np.zeros(BATCH_N_STATS)
    lib.ipm_run_instances(arr, n, _ptr(ns, ctypes.c_int), pp, qp, ctypes.byref(opt), ctypes.byref(bo),
                          int(mem_budget), sp, _ptr(it, ctypes.c_int), _ptr(er, ctypes.c_double),
                          _ptr(stt, ctypes.c_int), _ptr(stats, ctypes.c_double))
    return it, er, stt, dict(zip(BATCH_STATS, stats[:len(BATCH_STATS)])), states


class MLP:
    """The warm-start network of libipm.so (ipm_mlp_*).  Inputs and targets
    are device FP32 tensors; parameters and gradients travel as host FP32
    arrays in the logical layout (W1, b1, W2, b2, W3, b3)."""

    def __init__(self, d_in, d_hidden, d_out, max_batch=256, seed=0):
        self._lib = load()
        h = ctypes.c_void_p()
        st = self._lib.ipm_mlp_create(int(d_in), int(d_hidden), int(d_out), int(max_batch), int(seed),
                                      ctypes.byref(h))
        if st != IPM_OK:
            raise IPMError(st, "ipm_mlp_create failed")
        self._h = h
        self.d_in, self.d_hidden, self.d_out, self.max_batch = d_in, d_hidden, d_out, max_batch

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ipm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != IPM_OK:
            raise IPMError(st, what)

    @property
    def n_params(self):
        return int(self._lib.ipm_mlp_param_count(self._h))

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        self._check(self._lib.ipm_mlp_set_params(self._h, _ptr(p, ctypes.c_float)), "set_params")

    def get_params(self):
        p = np.empty(self.n_params, dtype=np.float32)
        self._check(self._lib.ipm_mlp_get_params(self._h, _ptr(p, ctypes.c_float)), "get_params")
        return p

    def set_normalization(self, in_mean, in_std, out_mean, out_std):
        a = [np.ascontiguousarray(v, dtype=np.float32) for v in (in_mean, in_std, out_mean, out_std)]
        self._check(self._lib.ipm_mlp_set_normalization(self._h, *[_ptr(v, ctypes.c_float) for v in a]),
                    "set_normalization")

    def forward(self, x, out=None, stream=None):
        import torch
        B = x.shape[0]
        if out is None:
            out = torch.empty((B, self.d_out), dtype=torch.float32, device=x.device)
        self._check(self._lib.ipm_mlp_forward(self._h, ctypes.c_void_p(x.data_ptr()), B,
                                              ctypes.c_void_p(out.data_ptr()), _stream(stream)), "forward")
        return out

    def gradients(self, x, t, stream=None):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float(0)
        self._check(self._lib.ipm_mlp_gradients(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                                x.shape[0], _ptr(g, ctypes.c_float), ctypes.byref(loss),
                                                _stream(stream)), "gradients")
        return loss.value, g

    def train_step(self, x, t, lr, stream=None):
        loss = ctypes.c_float(0)
        self._check(self._lib.ipm_mlp_train_step(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                                 x.shape[0], float(lr), ctypes.byref(loss), _stream(stream)),
                    "train_step")
        return loss.value
