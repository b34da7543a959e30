"""Multi-instance runner, CUDA-graph replay and autotuner (needs a GPU).

* graphs: a solve that replays the condensation as captured CUDA graphs
  gives bit-identical iterates to direct launches;
* autotuner: the tuned launch shapes change only the rounding of the
  scenario-group split (K_hat within 1e-12), the iteration count not at all;
* batch: independent instances of uneven sizes solved together (grouped
  persistent contraction, one stream per instance) give bit-identical
  results to solving each alone, and the small ones match the oracle;
* run_instances: the memory-budgeted create/solve/destroy runner returns the
  same states.
"""
import numpy as np
import pytest

from oracle import ipm as oipm
from oracle import opf
from paper_2301_04869_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_04869_gb300 import ipm
    ipm.load()
    return ipm


# (n_bus, n_gen, N, sigma, seed): uneven sizes and scenario counts, one ragged
# single-scenario case (each converges under the oracle in 18-26 iterations)
BATCH = [(30, 6, 1, 0.0, 0), (60, 9, 5, 0.05, 0), (100, 15, 8, 0.05, 3), (150, 22, 12, 0.05, 5),
         (200, 30, 3, 0.05, 7), (120, 18, 17, 0.05, 9), (1000, 150, 2, 0.05, 0)]
# (the 1000-bus instance needs more than the default 48 KB of shared memory
# per block in its solves, while the small ones do not)


def instances():
    out = []
    for n, ng, N, sig, seed in BATCH:
        net, pd, qd = synth.screened_network(n, ng, N, sig, seed=seed, scen_seed=seed + 1)
        out.append((net, pd, qd))
    return out


def solve_alone(gpu, net, pd, qd, **kw):
    sol = gpu.Solver(net, pd, qd, **kw)
    k, e = sol.ipm_solve()
    return k, e, sol.ipm_get_state()


def test_graph_replay_bit_identical(gpu):
    import torch
    net, pd, qd = instances()[1]
    k0, e0, s0 = solve_alone(gpu, net, pd, qd)
    st = torch.cuda.Stream()
    sol = gpu.Solver(net, pd, qd, graphs=True)
    with torch.cuda.stream(st):
        k1, e1 = sol.ipm_solve(stream=st)
        s1 = sol.ipm_get_state(stream=st)
    assert k1 == k0
    np.testing.assert_array_equal(s1, s0)
    _, launches = sol.timers()
    assert launches > 0


def test_graph_replay_mixed_bit_identical(gpu):
    import torch
    net, pd, qd = synth.workload("opf1000_n64", n_scen=4)
    a = gpu.Solver(net, pd, qd, precision=gpu.PREC_MIXED)
    ka, ea = a.ipm_solve()
    st = torch.cuda.Stream()
    b = gpu.Solver(net, pd, qd, precision=gpu.PREC_MIXED, graphs=True)
    with torch.cuda.stream(st):
        kb, eb = b.ipm_solve(stream=st)
    assert ka == kb
    np.testing.assert_array_equal(a.ipm_get_state(), b.ipm_get_state(stream=st))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_changes_rounding_only(gpu, precision):
    prec = gpu.PREC_FP64 if precision == "fp64" else gpu.PREC_MIXED
    net, pd, qd = synth.workload("opf1000_n64", n_scen=8)
    a = gpu.Solver(net, pd, qd, precision=prec)
    b = gpu.Solver(net, pd, qd, precision=prec, autotune=True)
    for s in (a, b):
        s.ipm_eval_derivatives()
        s.ipm_condense_scenarios()
    Ka, Kb = a.ipm_get_quantity(gpu.Q_KHAT), b.ipm_get_quantity(gpu.Q_KHAT)
    tol = 1e-12 if prec == gpu.PREC_FP64 else 1e-6
    assert np.abs(Ka - Kb).max() <= tol * np.abs(Ka).max()
    ka, _ = a.ipm_solve()
    kb, eb = b.ipm_solve()
    assert eb <= 1e-8
    assert abs(ka - kb) <= (0 if prec == gpu.PREC_FP64 else 2)


def test_batch_bit_identical_to_alone(gpu):
    insts = instances()
    alone = [solve_alone(gpu, *t) for t in insts]
    sols = [gpu.Solver(*t) for t in insts]
    it, er, st, stats = gpu.ipm_solve_batch(sols, n_threads=4, window_us=5000.0)
    assert (st == 0).all(), st
    assert stats["grouped_launches"] > 0
    assert stats["instances_per_launch"] > 1.0
    for j, (k, e, s) in enumerate(alone):
        assert it[j] == k, j
        assert er[j] <= 1e-8
        np.testing.assert_array_equal(sols[j].ipm_get_state(), s)


def test_batch_small_instances_match_oracle(gpu):
    insts = instances()[:2]
    sols = [gpu.Solver(*t) for t in insts]
    it, er, st, _ = gpu.ipm_solve_batch(sols, n_threads=2)
    assert (st == 0).all()
    for j, (net, pd, qd) in enumerate(insts):
        M = opf.Model(net, pd, qd)
        st_o, k_o, _ = oipm.solve(M)
        assert it[j] == k_o
        s = sols[j].split_state(sols[j].ipm_get_state())
        np.testing.assert_allclose(s["u"], st_o["u"], rtol=0, atol=1e-8)
        np.testing.assert_allclose(s["x"], st_o["x"], rtol=0, atol=1e-8)


def test_batch_ungrouped_and_graphs(gpu):
    """Without the grouped contraction, and with graphs, the same results."""
    insts = instances()[2:5] + instances()[6:]
    alone = [solve_alone(gpu, *t) for t in insts]
    for kw in (dict(group_contraction=False), dict(group_contraction=True)):
        sols = [gpu.Solver(*t, graphs=True) for t in insts]
        it, er, st, _ = gpu.ipm_solve_batch(sols, n_threads=3, **kw)
        assert (st == 0).all()
        for j, (k, e, s) in enumerate(alone):
            assert it[j] == k
            np.testing.assert_array_equal(sols[j].ipm_get_state(), s)


def test_run_instances_under_budget(gpu):
    insts = instances()
    alone = [solve_alone(gpu, *t) for t in insts]
    nets = [t[0] for t in insts]
    # a budget of ~2 instances' estimates forces admission in waves
    it, er, st, stats, states = gpu.ipm_run_instances(
        nets, [t[1] for t in insts], [t[2] for t in insts], mem_budget=200 << 20, n_threads=4,
        want_states=True)
    assert (st == 0).all(), st
    for j, (k, e, s) in enumerate(alone):
        assert it[j] == k
        np.testing.assert_array_equal(states[j], s)


def test_batch_rejects_bad_arguments(gpu):
    import ctypes
    lib = gpu.load()
    it = np.zeros(1, dtype=np.int32)
    er = np.zeros(1)
    stt = np.zeros(1, dtype=np.int32)
    hs = (ctypes.c_void_p * 1)(None)
    r = lib.ipm_solve_batch(hs, 1, None, None, it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            er.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            stt.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), None)
    assert r == 1  # IPM_ERR_ARG: null context
