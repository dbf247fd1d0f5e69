"""Oracle pins against the closed forms: Prop. 1 (Eq. (8)), Lemma 1 (Eq. (12)),
Theorems 1-2 (Eqs. (13), (16)), Eqs. (22)-(24), and the no-jump fidelity."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import core

EMPTY = core.History(cand_slice=[], cand_site=[], final_u=0.0)


def _final(p, gamma):
    _, d = core.run_one(p, 1, 0, gamma, EMPTY)
    return d


@pytest.mark.parametrize("n,k", [(2, 1), (2, 2), (3, 3), (4, 2), (5, 4), (6, 1), (8, 3)])
@pytest.mark.parametrize("gamma", [1e-5, 1e-3, 3e-2])
def test_qubit_good_branch_theorem2(n, k, gamma):
    """No jump: every branch ends as Eq. (16), exactly (to rounding)."""
    p = W.random_columns(W.QUBIT, n, k, D=min(1 << n, 7), seed=n * 31 + k)
    d = _final(p, gamma)
    want = {}
    for i, j, c in zip(p.addr, p.bus, p.amp):
        for word, A in cf.good_branch_qubit(int(i), int(j), int(p.memory[int(i)]), n, k, gamma).items():
            want[(int(i), word)] = c * A
    nrm = math.sqrt(sum(abs(v) ** 2 for v in want.values()))
    got = {}
    for a_, b_, cfg, amp in zip(d.addr, d.bus, d.configs, d.amp):
        assert cfg == ()                        # tree back in |0...0>
        got[(int(a_), int(b_))] = amp
    for key in set(got) | set(want):
        assert abs(got.get(key, 0.0) - want.get(key, 0.0) / nrm) < 1e-13


@pytest.mark.parametrize("n,k", [(3, 2), (5, 3)])
def test_hamming_collapse_fig3a(n, k):
    """Words of equal Hamming weight w = Ham(c xor b_out) share one probability."""
    gamma = 2e-2
    p = W.Problem(W.QUBIT, n, k, W.memory_bits(n, k, 4), np.array([5], np.uint32),
                  np.array([1], np.uint32), np.array([1.0 + 0j]))
    d = _final(p, gamma)
    b_out = 1 ^ int(p.memory[5])
    by_w = {}
    for b, amp in zip(d.bus, d.amp):
        by_w.setdefault(bin(int(b) ^ b_out).count("1"), []).append(abs(amp) ** 2)
    a = math.sqrt(1 - gamma)
    al, be = cf.alpha(a, 2 * n), cf.beta(a, 2 * n)
    z = (al * al + be * be) ** k
    for w, ps in by_w.items():
        assert max(ps) - min(ps) < 1e-15
        assert ps[0] == pytest.approx(al ** (2 * (k - w)) * be ** (2 * w) / z, rel=1e-11)


@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (3, 1), (4, 3), (6, 2)])
def test_qutrit_prop1(n, k):
    """Prop. 1 / Fig. 3(b): definite word j xor d_i, relative weights (1-gamma)^dc."""
    gamma = 7e-3
    p = W.random_columns(W.QUTRIT, n, k, D=min(1 << n, 6), seed=n + 100 * k)
    d = _final(p, gamma)
    want = {}
    for i, j, c in zip(p.addr, p.bus, p.amp):
        for word, A in cf.good_branch_qutrit(int(i), int(j), int(p.memory[int(i)]), n, k, gamma).items():
            want[(int(i), word)] = c * A
    nrm = math.sqrt(sum(abs(v) ** 2 for v in want.values()))
    got = {(int(a_), int(b_)): amp for a_, b_, amp in zip(d.addr, d.bus, d.amp)}
    assert all(cfg == () for cfg in d.configs)  # all-W tree
    assert set(got) == set(want)
    for key, v in want.items():
        assert abs(got[key] - v / nrm) < 1e-13


def test_lemma1_limits():
    for d in range(0, 12):
        assert cf.alpha(1.0, d) == 1.0 and cf.beta(1.0, d) == 0.0       # a = 1: ideal fetch
    for a in (0.3, 0.9, 0.999):
        assert cf.alpha(a, 0) == 1.0 and cf.beta(a, 0) == 0.0            # d = 0: identity
        for d in range(1, 9):                                             # norm = no-jump prob.
            assert cf.alpha(a, d) ** 2 + cf.beta(a, d) ** 2 == pytest.approx((1 + a ** (2 * d)) / 2, rel=1e-15)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 8])
def test_leakage_law_eq20(n):
    """Per-qubit wrong-bit probability of a no-jump branch, read off the
    oracle's evolved state, equals beta^2/(alpha^2+beta^2) and approaches
    n^2 gamma^2 / 4 with log-log slope 2 (Fig. 5(a))."""
    pts = []
    for gamma in [1e-5, 1e-4, 1e-3]:
        p = W.Problem(W.QUBIT, n, 1, W.memory_bits(n, 1, 8), np.array([3 % (1 << n)], np.uint32),
                      np.array([0], np.uint32), np.array([1.0 + 0j]))
        d = _final(p, gamma)
        b_out = int(p.memory[3 % (1 << n)])
        err = sum(abs(amp) ** 2 for b, amp in zip(d.bus, d.amp) if int(b) != b_out)
        assert err == pytest.approx(cf.leakage(gamma, n), rel=1e-7)
        pts.append((gamma, err))
    slope = (math.log(pts[-1][1]) - math.log(pts[0][1])) / (math.log(pts[-1][0]) - math.log(pts[0][0]))
    assert 1.99 < slope < 2.003
    assert pts[0][1] / cf.leakage_asymptote(pts[0][0], n) == pytest.approx(1.0, abs=1e-3)


@pytest.mark.parametrize("gamma", [1e-6, 1e-3, 0.05, 0.4])
@pytest.mark.parametrize("n", [1, 3, 7, 12])
def test_eq21_identity(gamma, n):
    lhs, rhs = cf.channel_error_split(gamma, n)
    assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-16)   # 1 - a^2n cancels at small gamma


@pytest.mark.parametrize("enc,n,k,gamma", [(W.QUBIT, 6, 1, 1e-3), (W.QUTRIT, 3, 1, 1e-3), (W.QUBIT, 4, 3, 5e-3)])
def test_no_jump_trajectories_equal_F0(enc, n, k, gamma):
    """Trajectories in which no jump fires all return the closed-form F0
    (the identical no-jump rows of Tab. III)."""
    p = W.data_loading(enc, n, k, seed=2001)
    r = core.run(p, 2001, 0, [gamma] * 300)
    F0 = cf.no_jump_fidelity(enc, n, k, gamma, p.addr, p.bus, p.amp, p.memory)
    nj = r[r["jumps"] == 0]
    assert len(nj) > 20
    assert np.all(nj["q_ground"] == 1)
    assert np.max(np.abs(nj["fidelity"] - F0)) < 1e-13


@pytest.mark.parametrize("n,k,gamma,wmax", [(6, 4, 1e-3, 0), (8, 3, 1e-4, 1), (10, 8, 1e-3, 2), (4, 2, 1e-2, 0)])
def test_low_weight_truncation_bound(n, k, gamma, wmax):
    """Sec. V cost discussion: each unit of Hamming weight costs beta/alpha
    = O(n gamma) in amplitude, so the words dropped at weight > w_max carry
    relative amplitudes at most (n gamma)^(w_max + 1), and the kept words'
    norm deficit is the binomial tail of the Eq. (13) amplitudes."""
    a = math.sqrt(1 - gamma)
    al, be = cf.alpha(a, 2 * n), cf.beta(a, 2 * n)
    assert be / al <= n * gamma
    top = cf.hamming_amplitude(0, 0, k, a, n)
    drop = [cf.hamming_amplitude(c, 0, k, a, n) for c in range(1 << k) if bin(c).count("1") > wmax]
    assert max(abs(x) for x in drop) / abs(top) <= (n * gamma) ** (wmax + 1)
    tail = sum(x * x for x in drop)
    want = sum(math.comb(k, w) * al ** (2 * (k - w)) * be ** (2 * w) for w in range(wmax + 1, k + 1))
    assert abs(tail - want) <= 1e-15 * max(1.0, want)
    total = sum(cf.hamming_amplitude(c, 0, k, a, n) ** 2 for c in range(1 << k))
    assert abs(total - (al * al + be * be) ** k) < 1e-14
