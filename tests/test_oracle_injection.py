"""Oracle pins from single-fault injection (Sec. III.B, Sec. VI.B) and from the
density-matrix cross-check of App. C (ensemble means)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import core, dm

N3, K3 = 3, 3


def _families(d, tol=1e-12):
    fam, bus = {}, {}
    for a, b, cfg, amp in zip(d.addr, d.bus, d.configs, d.amp):
        if abs(amp) < tol:
            continue
        fam.setdefault(int(a), set()).add(cfg)
        bus.setdefault(int(a), set()).add(int(b))
    return {a: frozenset(s) for a, s in fam.items()}, bus


def test_x_flip_family_divergence_eq9():
    """X flip at every (node, slot, slice) of the n=3, k=3 tree, no other
    noise: (i) addresses outside subtree(v) keep the ideal bus word; (ii) all
    addresses outside bad(v) of Eq. (9) share one final tree configuration;
    (iii) over slots and slices, the divergent set of each node reaches the
    boundary of bad(v)."""
    p = W.data_loading(W.QUBIT, N3, K3, seed=12)
    T = 6 * N3 + 2 * K3
    reach = {}
    for v in range(7):
        lo_s, hi_s = core.bad_range(W.QUTRIT, N3, v)     # subtree(v)
        lo_b, hi_b = core.bad_range(W.QUBIT, N3, v)      # bad(v), Eq. (9)
        reach[v] = set()
        for slot in (0, 1):
            for s in range(1, T):
                h = core.History([], [], final_u=0.0, flips=[(s, 2 * v + slot)])
                _, d = core.run_one(p, 1, 0, 0.0, h)
                fam, bus = _families(d)
                for i in range(8):
                    if not lo_s <= i < hi_s:
                        assert bus[i] == {int(p.memory[i])}
                if v == 0:
                    continue
                outside = [i for i in range(8) if not lo_b <= i < hi_b]
                ref = fam[outside[0]]
                assert all(fam[i] == ref for i in outside)
                reach[v] |= {i for i in range(8) if fam[i] != ref}
        if v:
            assert reach[v] <= set(range(lo_b, hi_b))
    # the boundary is reached for every node below the root
    for v in range(1, 7):
        lo_b, hi_b = core.bad_range(W.QUBIT, N3, v)
        assert reach[v] == set(range(lo_b, hi_b)), (v, reach[v])


def test_damping_fault_containment():
    """A fired damping jump at site q of node v leaves only addresses of
    subtree(v) (damping creates no strays; Sec. III.B)."""
    p = W.data_loading(W.QUBIT, N3, K3, seed=12)
    T = 6 * N3 + 2 * K3
    occ = core.occupancy(p)
    fired = 0
    for q in range(14):
        v = q >> 1
        lo, hi = core.bad_range(W.QUTRIT, N3, v)
        for s in range(1, T):
            if not occ[s, q]:
                continue
            h = core.History([s], [q], aux_u={s: 1.0 - 1e-12}, final_u=0.0)
            res, d = core.run_one(p, 1, 0, 0.05, h)
            assert res["jumps"] == 1 and res["first_jump_slice"] == s
            assert all(lo <= int(a) < hi for a in d.addr)
            fired += 1
    assert fired == 144


def _mc(enc, n, k, mem, gamma, N, seed):
    p = W.data_loading(enc, n, k, seed=1)
    p.memory = np.asarray(mem, np.uint8)
    r = core.run(p, seed, 0, [gamma] * N)
    return r


@pytest.mark.parametrize("enc,n,k,mem,gamma", [
    (W.QUBIT, 2, 1, [0, 1, 1, 0], 0.05),
    (W.QUBIT, 2, 1, [0, 1, 1, 0], 0.2),
    (W.QUBIT, 2, 2, [3, 1, 0, 2], 0.1),
    (W.QUTRIT, 1, 1, [1, 0], 0.1),
    (W.QUTRIT, 1, 1, [0, 1], 0.35),
])
def test_ensemble_mean_vs_density_matrix(enc, n, k, mem, gamma):
    F_rho, tr, _ = dm.simulate(enc, n, k, np.asarray(mem, np.uint8), gamma)
    assert abs(tr - 1) < 1e-12
    N = 40000
    r = _mc(enc, n, k, mem, gamma, N, seed=4242)
    for col in ("fidelity", "fidelity_unsampled"):
        m = r[col].mean()
        se = r[col].std() / math.sqrt(N)
        assert abs(m - F_rho) < 4.5 * se + 1e-12, (col, m, F_rho, se)


def test_output_distribution_vs_density_matrix():
    """Trajectory-averaged (address, bus) distribution vs the DM marginal."""
    mem = np.array([0, 1, 1, 0], np.uint8)
    gamma = 0.2
    _, _, marg = dm.simulate(W.QUBIT, 2, 1, mem, gamma)
    p = W.data_loading(W.QUBIT, 2, 1, seed=1)
    p.memory = mem
    N = 3000
    acc = {}
    for t in range(N):
        _, d = core.run_one(p, 77, t, gamma, None, cap=256)
        for a, b, amp in zip(d.addr, d.bus, d.amp):
            acc[(int(a), int(b))] = acc.get((int(a), int(b)), 0.0) + abs(amp) ** 2 / N
    keys = set(acc) | set(marg)
    tvd = 0.5 * sum(abs(acc.get(x, 0.0) - marg.get(x, 0.0)) for x in keys)
    assert tvd < 0.03
