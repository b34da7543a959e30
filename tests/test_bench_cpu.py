"""Host logic of bench.py (no GPU): the roofline entry picks the dominant
phase among those that are one kernel family and computes its fraction from
the work per launch; the emulated contraction's issued flops count the upper
tiles; the Clocks summary flags throttle reasons."""
import importlib.util
import os
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1600.0}


def dims(**kw):
    d = dict(n_scen=4, n_x=100, n_u=20, nnz_lu=1000, nnz_kx=300, nnz_ku=50, nd=0, big_block=0, lu_sparse_ops=500)
    d.update(kw)
    return SimpleNamespace(**d)


def phases(**ms):
    names = ("eval", "condense_K", "lu", "zsolve", "gemm", "reduced_rhs", "cholesky", "recover", "linesearch",
             "split", "fallback", "solve1")
    return {n: (ms.get(n, 0.0), 2.0 if n in ms else 0.0) for n in names}


def test_composite_phases_never_picked(bench):
    # recover, fallback, linesearch and reduced_rhs are sequences of kernels
    ph = phases(recover=900.0, fallback=5000.0, linesearch=800.0, reduced_rhs=700.0, zsolve=10.0, gemm=5.0)
    r = bench.roofline(ph, dims(), PEAKS, "measured", "mixed")
    assert r["kernel"].startswith("k_zsolve32")


def test_solve1_bytes_and_fraction(bench):
    d = dims()
    # two launches of 1 ms each: 8 (nnz_lu + 2 n_x) N bytes per launch
    r = bench.roofline(phases(solve1=2.0, zsolve=1.0), d, PEAKS, "measured", "mixed")
    byt = 8.0 * (d.nnz_lu + 2 * d.n_x) * d.n_scen
    assert r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(byt / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])


def test_zsolve_flops_per_precision(bench):
    d = dims()
    r64 = bench.roofline(phases(zsolve=2.0), d, PEAKS, "measured", "fp64")
    r32 = bench.roofline(phases(zsolve=2.0), d, PEAKS, "measured", "mixed")
    prod = 2.0 * (d.nnz_kx + d.nnz_ku) * d.n_u * d.n_scen
    assert r64["achieved"] * 1e12 * 1e-3 == pytest.approx(2.0 * d.nnz_lu * (d.n_u + 1) * d.n_scen + prod)
    assert r32["achieved"] * 1e12 * 1e-3 == pytest.approx(2.0 * d.nnz_lu * d.n_u * d.n_scen + prod)
    assert r64["peak"] == bench.FP64_PEAK_TFLOPS and r32["peak"] == bench.FP32_PEAK_TFLOPS


def test_lu_flops_with_dense_block(bench):
    d = dims(nd=10, big_block=1)
    r = bench.roofline(phases(lu=2.0), d, PEAKS, "measured", "mixed")
    flops = (2.0 * d.lu_sparse_ops + (2.0 / 3.0) * d.nd ** 3) * d.n_scen
    assert r["achieved"] == pytest.approx(flops / 1e-3 / 1e12)


def test_emu_issued_flops_upper_tiles(bench):
    # n_u = 128: one 128-row tile row and two 64-column tiles, both on or above the diagonal;
    # 512 contraction rows: 36 slice products of 2 x 512 x 128 x 64 flop each
    assert bench.emu_issued_flops(128, 512) == 36 * 2.0 * 512 * 128 * 64 * 2
    # n_u = 256: tile rows 0 (4 column tiles) and 1 (the 2 tiles from the diagonal on)
    assert bench.emu_issued_flops(256, 1) == 36 * 2.0 * 512 * 128 * 64 * 6


def test_clock_summary_reasons(bench):
    c = bench.Clocks()
    c.out = "0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active\n" \
            "0, 1900, 2070, 1380, 0x4, Not Active, Not Active, Not Active, Active\n"
    s = c.summary()
    assert s["sm_max_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"] and s["samples"] == 2
    c.out = ""
    assert c.summary()["sm_mhz"] is None
