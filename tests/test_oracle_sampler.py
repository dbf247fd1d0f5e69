"""Oracle pins for the noise sampler and the classifier: Philox4x32-10
against an independent implementation, the geometric gaps of the fault
stream against the inverse CDF, the candidate rate, Eq. (7), Eq. (9),
Eq. (25), and the probability that an address stays good."""
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import core

_TRITON_CHECK = r'''
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
from triton.language.random import philox
@triton.jit
def kern(c_ptr, k_ptr, o_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(c_ptr + 4 * i + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(c_ptr + 4 * i + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(c_ptr + 4 * i + 3).to(tl.uint32, bitcast=True)
    o0, o1, o2, o3 = philox(tl.load(k_ptr + i), c0, c1, c2, c3)
    tl.store(o_ptr + 4 * i + 0, o0.to(tl.int32, bitcast=True))
    tl.store(o_ptr + 4 * i + 1, o1.to(tl.int32, bitcast=True))
    tl.store(o_ptr + 4 * i + 2, o2.to(tl.int32, bitcast=True))
    tl.store(o_ptr + 4 * i + 3, o3.to(tl.int32, bitcast=True))
d = np.load(sys.argv[1])
ctr, keys = d["ctr"], d["keys"]
o = torch.zeros(ctr.size, dtype=torch.int32)
kern[(1,)](torch.from_numpy(ctr.view(np.int32).copy()), torch.from_numpy(keys.view(np.int64).copy()), o, N=len(keys))
np.save(sys.argv[2], o.numpy().view(np.uint32).reshape(-1, 4))
'''


def test_philox_against_independent_implementation(tmp_path):
    """Triton's Philox4x32-10 (its interpreter runs on the CPU) is written
    independently from the same published definition."""
    rng = np.random.default_rng(17)
    N = 64
    ctr = rng.integers(0, 2 ** 32, size=(N, 4), dtype=np.uint64).astype(np.uint32)
    keys = rng.integers(0, 2 ** 64, size=N, dtype=np.uint64)
    ctr[0], keys[0] = 0, 0
    ctr[1], keys[1] = 0xFFFFFFFF, 2 ** 64 - 1
    ctr[2] = [5, 2 | (1 << 24), 123, 0]                 # a FAULT-stream counter
    inp, out = tmp_path / "in.npz", tmp_path / "out.npy"
    np.savez(inp, ctr=ctr, keys=keys)
    script = tmp_path / "chk.py"
    script.write_text(_TRITON_CHECK)
    env = dict(os.environ, TRITON_INTERPRET="1")
    try:
        subprocess.run([sys.executable, str(script), str(inp), str(out)], check=True, env=env,
                       timeout=300, capture_output=True)
    except Exception as e:                               # pragma: no cover
        pytest.skip(f"triton interpreter unavailable: {e}")
    ref = np.load(out)
    for r in range(N):
        assert core.philox(ctr[r], int(keys[r])) == [int(x) for x in ref[r]]


def test_threshold_exact():
    for g in [1e-5, 1e-3, 0.0123, 0.2, 0.5, 2.0 ** -60, 0.0]:
        assert core.threshold(g) == math.floor(Fraction(g) * 2 ** 64)


@pytest.mark.parametrize("gamma", [1e-5, 3e-4, 0.01, 0.2, 0.6])
def test_gap_is_geometric_inverse_cdf(gamma):
    """The fault stream's gap of a uniform word u is the inverse CDF of the
    geometric law: the largest j with (1 - gamma)^j > u / 2^64, capped at
    2^13 - 1.  The fixed-point powers carry an absolute error of a few
    2^-64 per factor, so the bracket (1-gamma)^(g+1) <= u/2^64 < (1-gamma)^g
    is checked with an absolute slack of 1e-14 in probability."""
    rng = np.random.default_rng(int(gamma * 1e6) + 3)
    words = [int(x) for x in rng.integers(0, 2 ** 64, size=400, dtype=np.uint64)]
    words += [0, 1, 2 ** 63, 2 ** 64 - 1, 2 ** 64 - 2 ** 20]
    q = 1.0 - gamma
    eps = 1e-14
    for u in words:
        v = u / 2.0 ** 64
        g = core.gap(u, gamma)
        assert q ** g > v - eps, (u, g)
        if g < 2 ** 13 - 1:
            assert q ** (g + 1) <= v + eps, (u, g)
        else:
            assert q ** g <= 2.0 * (v + eps) or q ** (2 ** 13) < 1e-300 or v < q ** (2 ** 13) + eps
    # gamma = 1/2, where the powers are exact: acc starts at 2^64 - 1, so the
    # first boundary sits at floor((2^64 - 1) / 2) = 2^63 - 1
    for u, want in [(2 ** 63, 0), (2 ** 63 - 1, 0), (2 ** 63 - 2, 1), (2 ** 62 - 1, 1), (2 ** 62 - 2, 2)]:
        assert core.gap(u, 0.5) == want
    assert core.gap(12345, 0.0) == 0xFFFFFFFF                # no candidates at all


def test_gap_law_small_gamma_mean():
    """Mean gap over a stream of words against 1/gamma - 1 (truncated law)."""
    gamma = 0.05
    rng = np.random.default_rng(9)
    g = np.array([core.gap(int(u), gamma) for u in rng.integers(0, 2 ** 64, size=20000, dtype=np.uint64)])
    q = 1 - gamma
    want = q / gamma                                          # E[G], tail beyond 8191 negligible
    assert abs(g.mean() - want) < 5 * math.sqrt(q) / gamma / math.sqrt(len(g))


def test_candidate_rate_binomial():
    n, k, gamma = 6, 2, 0.01
    p = W.data_loading(W.QUBIT, n, k, seed=1)
    tot = 0
    trials = 0
    for t in range(40):
        sl, st, _, _, _ = core.sample_faults(p, 99, t, gamma)
        tot += len(sl)
        trials += 2 * ((1 << n) - 1) * (cf.slices(n, k) - 1)
        assert np.all(np.diff(sl) >= 0)
    mean = trials * gamma
    sd = math.sqrt(trials * gamma * (1 - gamma))
    assert abs(tot - mean) < 5 * sd


@pytest.mark.parametrize("n", range(2, 13))
def test_mark_sources_eq22(n):
    tot = 0
    for v in range((1 << n) - 1):
        lo, hi = core.bad_range(W.QUBIT, n, v)
        tot += hi - lo
    assert Fraction(tot, 1 << n) == Fraction(n) + Fraction((n - 1) * (n - 2), 4)
    # the qutrit subtree rule (Eq. (7)) gives n marking sources per address
    tot = sum(np.subtract(*core.bad_range(W.QUTRIT, n, v)[::-1]) for v in range((1 << n) - 1))
    assert tot == n << n


def test_bad_range_eq7_eq9_small_tree():
    """n = 3: Eq. (7) ranges and the Eq. (9) recursion, node by node."""
    n = 3
    sub = {v: core.bad_range(W.QUTRIT, n, v) for v in range(7)}
    assert sub[0] == (0, 8) and sub[1] == (0, 4) and sub[2] == (4, 8)
    assert [sub[v] for v in range(3, 7)] == [(0, 2), (2, 4), (4, 6), (6, 8)]
    bad = {v: core.bad_range(W.QUBIT, n, v) for v in range(7)}
    assert bad[0] == (0, 8)
    assert bad[1] == (0, 4) and bad[2] == (4, 8)           # children of the root
    assert bad[4] == sub[4] and bad[6] == sub[6]           # right children
    assert bad[3] == bad[1] and bad[5] == bad[2]           # left child -> parent


def test_classification_union_and_reference():
    p = W.random_columns(W.QUBIT, 7, 2, D=90, seed=5)
    for t in range(6):
        sl, st, bad, B, ref = core.sample_faults(p, 7, t, 2e-3)
        want = np.zeros(1 << 7, np.uint8)
        for q in st:
            lo, hi = core.bad_range(W.QUBIT, 7, int(q) >> 1)
            want[lo:hi] = 1
        assert np.array_equal(bad, want)
        isbad = want[p.addr]
        assert B == int(isbad.sum())
        goods = np.nonzero(isbad == 0)[0]
        assert ref == (int(goods[0]) if len(goods) else -1)


def test_p_good_closed_form():
    """P(address i good) = (1-gamma)^(2(T-1) * #{v : i in bad(v)})."""
    n, k, gamma = 4, 1, 4e-3
    p = W.data_loading(W.QUBIT, n, k, seed=1)
    src = np.zeros(1 << n, int)
    for v in range((1 << n) - 1):
        lo, hi = core.bad_range(W.QUBIT, n, v)
        src[lo:hi] += 1
    N = 3000
    good = np.zeros(1 << n)
    for t in range(N):
        _, _, bad, _, _ = core.sample_faults(p, 31, t, gamma)
        good += 1 - bad
    for i in range(1 << n):
        pg = cf.p_good(int(src[i]), gamma, n, k)
        assert abs(good[i] / N - pg) < 5 * math.sqrt(pg * (1 - pg) / N)
