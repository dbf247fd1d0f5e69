"""The product form of the data qubits (qubit encoding, damping): between
the first Hadamard wall and the return of the last data qubit (slices
2n+1 .. 4n+2k-1) one component stands for the 2^k wall configurations of a
branch (Lemma 1).  Fixed fault histories put candidates where the form has
to change:

- on a router that a data qubit passed on its way down: after the jump the
  router points the other way, the qubit is stranded below it on its way up
  and later meets a router swap of the unload, so the component goes
  explicit at the epoch boundary before that swap;
- on the data slot a data qubit sits in: the jump fixes that qubit (only the
  configurations with it excited survive);
- around slice 4n+2k-1, where the form becomes a binomial group or its
  explicit configurations.

Trajectories and final amplitudes against the oracle in both modes: integer
outputs bit-exact, floating point within 1e-12."""
import numpy as np
import pytest

import workloads as W
from oracle import core

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _node(i, n, L):
    """node of layer L on the path of address i (heap order)"""
    return (1 << L) - 1 + (i >> (n - L))


def _histories(p, n, k, ntraj, seed):
    """(slice, site) lists aimed at the changes of the product form"""
    rng = np.random.default_rng(seed)
    T, sU = 6 * n + 2 * k, 4 * n + 2 * k - 1
    M = 2 * ((1 << n) - 1)
    out = []
    for _ in range(ntraj):
        ev = set()
        for _ in range(2):
            a = int(p.addr[rng.integers(0, len(p.addr))])
            t = int(rng.integers(0, k))
            L = int(rng.integers(max(1, n - 3), n - 1))
            # the router of layer L after data qubit t passed it going down
            # (layer L -> L + 1 at 2n+2t+L+2) and before it comes back up
            # (layer L + 1 -> L at 4n+2t-L)
            lo, hi = 2 * n + 2 * t + L + 2, 4 * n + 2 * t - L - 1
            if lo <= hi:
                ev.add((int(rng.integers(lo, hi + 1)), 2 * _node(a, n, L)))
            # the data slot data qubit t reaches at layer L going down, or a leaf data slot later
            ev.add((2 * n + 2 * t + 1 + L, 2 * _node(a, n, L) + 1))
            ev.add((int(rng.integers(3 * n + 1, sU + 1)), 2 * _node(a, n, n - 1) + 1))
        for s in (sU - 1, sU, sU + 1):
            if rng.random() < 0.5:
                ev.add((s, int(rng.integers(0, M))))
        for _ in range(2):
            ev.add((int(rng.integers(1, T)), int(rng.integers(0, M))))
        out.append(sorted(ev))
    return out


def _set(sim, hists):
    cand, off = [], [0]
    for h in hists:
        cand += [(s << 16) | q for s, q in h]
        off.append(len(cand))
    sim.set_fault_history(torch.tensor(np.array(cand, np.int64).astype(np.int32), device="cuda:0"),
                          torch.tensor(np.array(off, np.int32), device="cuda:0"))


CASES = [
    (6, 3, "rand", 4), (6, 3, "rand", 13), (5, 2, "rand", 6), (7, 4, "rand", 9), (6, 4, "load", 0),
]


def _problem(n, k, kind, D, seed):
    if kind == "load":
        return W.data_loading(W.QUBIT, n, k, seed=seed)
    return W.random_columns(W.QUBIT, n, k, D=D, seed=seed)


@pytest.mark.parametrize("n,k,kind,D", CASES)
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_product_form_trajectories(n, k, kind, D, mode):
    from paper_2609_34935_b300 import QramSim
    seed = 4400 + 17 * n + k + D
    p = _problem(n, k, kind, D, seed)
    hists = _histories(p, n, k, 60, seed)
    sim = QramSim(p, seed=seed, device=0)
    _set(sim, hists)
    g = np.full(len(hists), 0.03)
    got = sim.results(sim.run(mode, 0, torch.tensor(g, device="cuda:0")))
    sim.set_fault_history()
    sim.close()
    data_phase = 0
    for t, h in enumerate(hists):
        r, _ = core.run_one(p, seed, t, 0.03, core.History([s for s, _ in h], [q for _, q in h]), cap=1 << 16)
        assert got["status"][t] == 0, t
        for f in ("jumps", "first_jump_slice", "jump_sites", "q_ground", "bad", "ref"):
            assert int(got[f][t]) == int(r[f]), (t, f)
        for f in ("fidelity", "fidelity_unsampled", "p_ground"):
            assert abs(got[f][t] - r[f]) < TOL, (t, f)
        data_phase += int(2 * n < r["first_jump_slice"] < 4 * n + 2 * k - 1)
    if kind == "rand":
        assert data_phase >= 5


def _hash_cfg(cfg):
    if not cfg:
        return 0
    h = 1469598103934665603
    for q, lv in cfg:
        v = (q << 2) | lv
        for b in range(4):
            h ^= (v >> (8 * b)) & 0xFF
            h = (h * 1099511628211) & (2 ** 64 - 1)
    return h or 1


@pytest.mark.parametrize("n,k,kind,D", [(6, 3, "rand", 4), (5, 3, "rand", 7)])
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_product_form_amplitudes(n, k, kind, D, mode):
    from paper_2609_34935_b300 import QramSim
    seed = 4600 + 17 * n + k + D
    p = _problem(n, k, kind, D, seed)
    hists = _histories(p, n, k, 12, seed)
    sim = QramSim(p, seed=seed, device=0)
    jumped = 0
    for t, h in enumerate(hists):
        hist = core.History([s for s, _ in h], [q for _, q in h])
        r, d = core.run_one(p, seed, t, 0.03, hist, cap=1 << 16)
        jumped += int(r["jumps"]) > 0
        want = {}
        for a, b, cfg, amp in zip(d.addr, d.bus, d.configs, d.amp):
            key = (int(a), int(b), _hash_cfg(cfg))
            want[key] = want.get(key, 0) + amp
        _set(sim, [h])                           # the dump runs history 0 with trajectory t's draws
        ga, gb, gh, gz = sim.dump_state(mode, t, 0.03)
        got = {}
        for a, b, hh, z in zip(ga, gb, gh, gz):
            key = (int(a), int(b), int(hh))
            got[key] = got.get(key, 0) + z
        for key in set(want) | set(got):
            assert abs(want.get(key, 0) - got.get(key, 0)) < TOL, (t, key)
    sim.set_fault_history()
    sim.close()
    assert jumped >= 3
