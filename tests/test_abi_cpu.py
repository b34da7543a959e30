"""C-ABI checks that need no GPU: the library loads, exports every entry
point declared in include/ipm.h, and rejects invalid arguments before it
touches the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2301_04869_gb300 import ipm, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(ipm_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(ipm.LIB_PATH):
        from paper_2301_04869_gb300 import build
        build.build()
    return ipm.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"ipm_eval_derivatives", "ipm_condense_scenarios", "ipm_factor_schur",
            "ipm_solve_kkt", "ipm_step"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_default_options(lib):
    o = ipm.Options()
    assert lib.ipm_default_options(ctypes.byref(o)) == 0
    assert o.tol == 1e-8 and o.max_iter == 200 and o.precision == ipm.PREC_FP64
    assert o.lu_pair == 1 and o.graphs == 0 and o.autotune == 0 and o.poison == 0
    assert o.tc_solve == 1


@pytest.mark.parametrize("field,value", [("precision", 3), ("solve_threads", 64), ("graphs", 2), ("autotune", -1),
                                         ("poison", 2), ("lu_pair", 2), ("tol", 0.0), ("max_iter", -1),
                                         ("tc_solve", 2)])
def test_rejects_bad_options(lib, field, value):
    """Invalid options are rejected before the device is touched."""
    net = synth.make_network(30, 6, seed=0)
    pd, qd = synth.make_scenarios(net, 2, 0.05, seed=1)
    o = ipm.Options()
    lib.ipm_default_options(ctypes.byref(o))
    setattr(o, field, value)
    keep, cnet = ipm._cnet(net)
    h = ctypes.c_void_p()
    pd = np.ascontiguousarray(pd)
    qd = np.ascontiguousarray(qd)
    st = lib.ipm_create(ctypes.byref(cnet), pd.shape[0], pd.ctypes.data_as(ipm._D), qd.ctypes.data_as(ipm._D),
                        ctypes.byref(o), ctypes.byref(h))
    assert st == 1 and not h.value  # IPM_ERR_ARG


def test_symbolic_export_rejects_bad_ids(lib):
    net = synth.make_network(30, 6, seed=0)
    keep, cnet = ipm._cnet(net)
    n = ctypes.c_longlong(0)
    assert lib.ipm_symbolic_export(ctypes.byref(cnet), -1, None, 0, ctypes.byref(n)) == 1
    assert lib.ipm_symbolic_export(ctypes.byref(cnet), len(ipm.SYM_NAMES), None, 0, ctypes.byref(n)) == 1
    assert lib.ipm_symbolic_export(None, 0, None, 0, ctypes.byref(n)) == 1
    assert lib.ipm_symbolic_export(ctypes.byref(cnet), 0, None, 0, ctypes.byref(n)) == 0 and n.value == 9


def _create(lib, net, pd, qd):
    k = dict(fr=net.fr.astype(np.int32), to=net.to.astype(np.int32), gen=net.gen_bus.astype(np.int32))
    c = ipm.Network(net.n_bus, net.n_line, net.n_gen,
                    k["fr"].ctypes.data_as(ipm._I), k["to"].ctypes.data_as(ipm._I), k["gen"].ctypes.data_as(ipm._I),
                    *[np.ascontiguousarray(getattr(net, a)).ctypes.data_as(ipm._D)
                      for a in ("r", "x", "b", "pmax", "qmax", "c2", "c1", "vmin", "vmax")])
    h = ctypes.c_void_p()
    pd = np.ascontiguousarray(pd)
    qd = np.ascontiguousarray(qd)
    st = lib.ipm_create(ctypes.byref(c), pd.shape[0], pd.ctypes.data_as(ipm._D), qd.ctypes.data_as(ipm._D),
                        None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("bad", ["nan_load", "neg_load", "zero_scen"])
def test_rejects_bad_loads(lib, bad):
    net = synth.make_network(30, 6, seed=0)
    pd, qd = synth.make_scenarios(net, 2, 0.05, seed=1)
    if bad == "nan_load":
        pd[1, 3] = np.nan
    elif bad == "neg_load":
        pd[0, 5] = -0.1
    else:
        pd = pd[:0]
        qd = qd[:0]
    st, h = _create(lib, net, pd, qd)
    assert st == 1 and not h.value  # IPM_ERR_ARG, nothing allocated


def test_null_context_calls(lib):
    assert lib.ipm_step(None, None, None, None) == 1
    assert lib.ipm_destroy(None) == 1
    assert lib.ipm_last_error(None) == b"null context"
