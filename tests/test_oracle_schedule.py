"""Oracle pins for the time-sliced schedule (Sec. II.A, Eqs. (2)-(4), Eq. (14),
Sec. VI.B injection count, App. C Tab. IV)."""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import core, dm

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))
EMPTY = core.History(cand_slice=[], cand_site=[], final_u=0.0)


@pytest.mark.parametrize("n", range(1, 15))
def test_schedule_slots_disjoint(n):
    for k in range(1, min(n, 4) + 1):
        assert core.schedule_rc(n, k) == core.OK
    assert core.schedule_rc(n, n + 1) == core.E_ARG      # k <= n is required


@pytest.mark.parametrize("n,k", [(2, 1), (3, 3), (5, 2), (12, 4)])
def test_event_times_eq4(n, k):
    sched = core.schedule(n, k)
    T = cf.slices(n, k)
    assert max(s for s, _, _ in sched) == T - 1
    bus = sorted((s, p) for s, g, p in sched if g == "bus")
    for t in range(k):
        assert (cf.tau_in(n, t), t) in bus and (cf.tau_out(n, t), t) in bus
        assert (cf.tau_fetch(n, t), "fetch", t) in sched
        assert cf.tau_out(n, t) - cf.tau_in(n, t) == 2 * n                       # Eq. (4) window
        assert cf.tau_out(n, t) == T - cf.tau_in(n, k - 1 - t)                   # mirror
    assert sorted(s for s, g, _ in sched if g in ("load", "unload")) == \
        sorted([2 * l + 1 for l in range(n)] + [T - 2 * l - 1 for l in range(n)])


@pytest.mark.parametrize("n", range(1, 15))
def test_data_qubits_never_meet_a_router_swap(n):
    """No router/data swap of a layer fires while a data qubit is in that
    layer.  Every item moves one layer per slice whatever its path, so this
    holds on and off the path: a data qubit's value never reaches a router,
    and its position depends on the routers alone (the schedule of Sec. II,
    data windows of Eq. (4))."""
    for k in range(1, n + 1):
        sched = core.schedule(n, k)
        layers = {}                                  # slice -> layers holding a data qubit after its gates
        for t in range(k):
            tin, tf, tout = cf.tau_in(n, t), cf.tau_fetch(n, t), cf.tau_out(n, t)
            for s in range(tin, tout):
                L = s - tin if s < tf else (n - 1 if s == tf else n - 1 - (s - tf))
                layers.setdefault(s, set()).add(L)
        swaps = [(s, L) for s, g, L in sched if g == "iswap"]
        assert len(swaps) == 2 * n
        for s, L in swaps:
            assert L not in layers.get(s - 1, set()) and L not in layers.get(s, set()), (n, k, s, L)


def test_injection_count_sec5b():
    g = GOLD["single_fault_injection"]
    p = W.data_loading(W.QUBIT, g["n"], g["k"], seed=3)
    occ = core.occupancy(p)
    T = cf.slices(g["n"], g["k"])
    M = 2 * ((1 << g["n"]) - 1)
    assert M == g["positions"] and T - 1 == g["slices"]
    total = (T - 1) * M
    assert total == g["damping_cases"] and 2 * total == g["cases"]
    nonvac = int(occ[1:T].sum())
    assert total - nonvac == g["vacuous"]


def test_dm_crosscheck_values_tab4():
    g = GOLD["dm_crosscheck"]
    mem = np.array(g["memory"], np.uint8)
    for row in g["rows"]:
        F, tr, _ = dm.simulate(W.QUBIT, g["n"], g["k"], mem, row["gamma"])
        assert abs(tr - 1.0) < 1e-12
        assert round(F, 4) == row["F_rho"]


def test_noise_free_equals_ideal():
    """gamma = 0: the final state is exactly the oracle map of Eq. (1)."""
    for enc in (W.QUTRIT, W.QUBIT):
        for n, k in [(1, 1), (2, 2), (3, 1), (4, 3), (5, 2)]:
            p = W.random_columns(enc, n, k, D=max(1, (1 << n) - 3), seed=11 * n + k)
            res, d = core.run_one(p, 5, 0, 0.0, EMPTY)
            assert res["fidelity"] == pytest.approx(1.0, abs=1e-14)
            want = {(int(i), int(j) ^ int(p.memory[int(i)])): complex(c) for i, j, c in zip(p.addr, p.bus, p.amp)}
            got = {(int(a), int(b)): amp for a, b, cfg, amp in zip(d.addr, d.bus, d.configs, d.amp)}
            assert all(len(cfg) == 0 for cfg in d.configs)
            for key in set(got) | set(want):           # wall merges leave ~1e-17 residues
                assert abs(got.get(key, 0.0) - want.get(key, 0.0)) < 1e-14


@pytest.mark.parametrize("n,k", [(2, 1), (3, 2), (4, 4), (6, 1)])
def test_address_window_eq12(n, k):
    """A single qubit-encoding branch with no candidates ends with norm
    a^(2 c_addr(i)) ((1+a^4n)/2)^k: address bit t damped for T-4t-2 layers
    (Eq. (14)), every data qubit for exactly 2n (Eq. (4))."""
    gamma = 0.013
    a = math.sqrt(1 - gamma)
    for i in [0, 1, (1 << n) - 1, (1 << n) // 3]:
        p = W.Problem(W.QUBIT, n, k, W.memory_bits(n, k, 9), np.array([i], np.uint32),
                      np.array([0], np.uint32), np.array([1.0 + 0j]))
        # fixed empty history: no jump, but K0 acts in every layer.  The oracle
        # renormalises, so compare the word distribution and, via a two-branch
        # input, the relative norm.
        q = W.Problem(W.QUBIT, n, k, p.memory, np.array([i, (i + 1) % (1 << n)], np.uint32),
                      np.array([0, 0], np.uint32), np.array([1, 1], np.complex128) / math.sqrt(2))
        _, d = core.run_one(q, 1, 0, gamma, EMPTY)
        w = {}
        for ad, amp in zip(d.addr, d.amp):
            w[int(ad)] = w.get(int(ad), 0.0) + abs(amp) ** 2
        j = (i + 1) % (1 << n)
        ratio = w[i] / w[j]
        want = a ** (2 * (cf.c_addr(i, n, k) - cf.c_addr(j, n, k)))
        assert ratio == pytest.approx(want, rel=1e-12)
