"""Host-side logic that needs no GPU: the synthetic input generators of the
newer workloads and the bench's bookkeeping (groups of the mixing workload,
the polynomial path's flop count)."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import poly as P
from paper_2606_20519_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_orthonormal_columns_and_scs_problem():
    rng = W.rng_for(1)
    B = W.orthonormal_columns(rng, 300, 25)  # rows of B are the columns of A
    np.testing.assert_allclose(B @ B.T, np.eye(25), atol=1e-14)
    At, b, c, u, v = W.scs_problem(n=12, k=7)
    m = 12 * 13 // 2
    assert At.shape == (7, m) and b.shape == (m,) and c.shape == (7,)
    assert u.shape == v.shape == (7 + m + 1,) and u[-1] == 1.0 and v[-1] == 1.0
    np.testing.assert_allclose(At @ At.T, np.eye(7), atol=1e-14)
    # seeded: the same call gives the same problem
    At2, b2, _, _, _ = W.scs_problem(n=12, k=7)
    np.testing.assert_array_equal(At, At2)
    np.testing.assert_array_equal(b, b2)


def test_mixing_workload_groups():
    wl = _bench().Workload("mixing")
    sides = wl.calls[0][1]
    g = wl.groups
    assert g[0] == 0 and g[-1] == len(sides) and all(g[i] < g[i + 1] for i in range(len(g) - 1))
    assert len(wl.nu) == len(g) - 1
    for q in range(len(g) - 1):
        blk = sides[g[q]:g[q + 1]]
        assert len(set(blk)) == 1  # one side per group
        n = blk[0]
        if len(blk) == 2:  # two outcomes of an instrument block of side d^2
            d = round(n ** 0.5)
            assert d * d == n and wl.nu[q] == pytest.approx(1.0 / (2 * d))
        else:  # a process block mixed with gamma * 1
            assert len(blk) == 1 and wl.nu[q] == pytest.approx(1.0 / n)
    assert wl.eps == 1e-16


def test_poly_roofline_flop_count():
    bench = _bench()

    class FakeLib:
        FP64 = 0
        SPLIT_TF32 = 1

        @staticmethod
        def poly_schedule(lo, steps=0):
            a, b, lk = P.poly_coeffs(lo, steps)
            return np.array(a), np.array(b), lk

    class Args:
        poly_lo = 1e-9

    class Wl:
        calls = [(None, [625]), (None, [4096, 4096])]

    K = len(P.poly_coeffs(1e-9)[0])
    roof, info = bench.poly_roofline(FakeLib, Args, Wl, 1.0, FakeLib.FP64)
    want = sum(K * 2.0 * n ** 3 + float(n) ** 3 for n in (625, 4096, 4096))
    assert roof["flops_per_step"] == pytest.approx(want, rel=1e-12)
    assert info["steps"] == K == 29
    roof_s, _ = bench.poly_roofline(FakeLib, Args, Wl, 1.0, FakeLib.SPLIT_TF32)
    assert roof_s["bound"] == "tensor" and roof_s["achieved"] == pytest.approx(8.0 * want / 1e-3 / 1e12)


def test_reference_arm_json_contract():
    """bench.py --impl reference times the oracle and prints one JSON line
    with the contract's keys (no GPU needed)."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config",
                          "single81", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["unit"] == "projections/s"


def test_binding_lists_every_declared_entry_point():
    import re
    from paper_2606_20519_gb300 import _lib
    text = open(os.path.join(ROOT, "include", "scs_psd.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int32_t|int64_t|const char\*)\s+(scs_psd_\w+)\s*\(", text, re.M))
    missing = declared - set(_lib.EXPORTS)
    assert not missing, sorted(missing)


def test_spectrum_recipes_match_the_documented_workloads():
    """The spectra are what the input table states (counts and ranges)."""
    rng = W.rng_for(5)
    s = W.spectrum_plain(rng, 81)
    assert (s > 0).sum() == 40 and (s < 0).sum() == 40 and (s == 0).sum() == 1
    assert s[s > 0].min() >= 0.1 and s[s > 0].max() <= 2.0 and s[s < 0].max() <= -0.1
    s = W.spectrum_admm(rng, 625)
    assert s.size == 625
    tiny, pos, neg = s[:300], s[300:500], s[500:]
    assert np.abs(tiny).max() < 1e-5 and pos.min() >= 0.01 and pos.max() <= 1.0 and neg.max() <= -0.01
    assert neg.size == 125
    s = W.spectrum_precision(rng, 4096)
    assert s.size == 4096 and np.abs(s[:2048]).max() <= 1.0 and np.abs(s[2048:3072]).max() < 1e-6
    big = np.abs(s[3072:])
    assert big.min() >= 1e-4 and big.max() <= 100.0
    s = W.spectrum_vjp(rng, 1296)
    assert (s == 1e-9).sum() == 65 and (s == -1e-9).sum() == 65
    b = W.uneven_batch(restarts=2)
    assert list(b.sides[:15]) == [4, 4, 9, 9, 16, 16, 25, 25, 36, 36, 49, 49, 64, 64, 625]
    assert b.sides[29] == 1296 and b.count == 30


def test_autograd_store_or_recompute_decision():
    from paper_2606_20519_gb300 import _lib
    from paper_2606_20519_gb300.autograd import stores_eigenpairs
    sides = [625, 81]
    nv, nl = _lib.eig_sizes(sides)
    assert (nv, nl) == (625 * 625 + 81 * 81, 706)
    need = 8 * (nv + nl)
    assert stores_eigenpairs(sides)  # no options: keep
    assert stores_eigenpairs(sides, _lib.make_opts(mem_budget_bytes=need))
    assert not stores_eigenpairs(sides, _lib.make_opts(mem_budget_bytes=need - 1))
    assert not stores_eigenpairs(sides, _lib.make_opts(recompute=1))
    assert stores_eigenpairs(sides, _lib.make_opts(recompute=2, mem_budget_bytes=1))
