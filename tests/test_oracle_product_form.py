"""After a fired router jump, the data qubits stay in product form.

Every item moves one layer per slice whatever its path, and no router/data
swap of a layer fires while a data qubit is in that layer, so a data qubit's
value never reaches a router.  After a jump that resets a router, a
surviving branch's 2^k data configurations (the first Hadamard wall's
components) therefore share one address part and one set of (perturbed)
data-qubit paths, and each data qubit t with value 1 is damped on every
slice it spends in the tree: the window of Eq. (4), whatever its path.  Between the
walls the configuration weights of a branch are then C_i * prod_t a^(2 m_t c_t),
m_t = the slices of that window up to the observation point.  The oracle
evolves every configuration explicitly; this checks its state against that
form."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import core


def _window(n, t, s_stop):
    """Damping layers data qubit t has spent in the tree after slice s_stop."""
    lo, hi = cf.tau_in(n, t), min(s_stop, cf.tau_out(n, t) - 1)
    return max(0, hi - lo + 1)


@pytest.mark.parametrize("n,k,s_stop", [(3, 2, 12), (3, 2, 14), (4, 3, 17)])
def test_post_jump_configuration_weights_factorise(n, k, s_stop):
    gamma = 0.1
    a2 = 1.0 - gamma
    p = W.data_loading(W.QUBIT, n, k, seed=7)
    # a candidate on the root router (site 0) while it holds the routed
    # address bit, drawn so that the jump fires: the survivors are the
    # branches whose top address bit is 1, and the root then routes left
    s_jump = 5
    assert s_stop < 4 * n + 2 * k - 1                # observed before the second wall
    h = core.History(cand_slice=[s_jump], cand_site=[0], aux_u={s_jump: 0.999}, final_u=0.5, stop_slice=s_stop)
    out, d = core.run_one(p, 7, 0, gamma, hist=h)
    assert out["jumps"] == 1 and out["first_jump_slice"] == s_jump
    m = [_window(n, t, s_stop) for t in range(k)]
    # expected weights relative to the heaviest configuration, one per value word c
    expect = sorted((a2 ** sum(m[t] for t in range(k) if (c >> t) & 1) for c in range(1 << k)), reverse=True)
    by = {}
    for i, amp in zip(d.addr, d.amp):
        by.setdefault(int(i), []).append(abs(amp) ** 2)
    assert sorted(by) == list(range(1 << (n - 1), 1 << n))      # top address bit 1
    for i, w in by.items():
        assert len(w) == 1 << k, (i, len(w))
        w = sorted(w, reverse=True)
        rel = [x / w[0] for x in w]
        assert np.allclose(rel, expect, rtol=1e-12, atol=0), (i, rel, expect)


@pytest.mark.parametrize("s_stop", [12, 14])
def test_jump_on_a_data_site_fixes_that_qubit(s_stop):
    """A jump that fires on the site of data qubit 0 keeps the configurations
    with c_0 = 1 and leaves that qubit at 0: each surviving branch keeps
    2^(k-1) configurations, weighted by the other qubits' windows alone."""
    n, k, gamma = 3, 2, 0.1
    a2 = 1.0 - gamma
    p = W.data_loading(W.QUBIT, n, k, seed=7)
    t0 = cf.tau_in(n, 0)                 # data qubit 0 has just entered d_0 (site 1)
    h = core.History(cand_slice=[5, t0], cand_site=[0, 1], aux_u={5: 0.999, t0: 0.999}, final_u=0.5,
                     stop_slice=s_stop)
    out, d = core.run_one(p, 7, 0, gamma, hist=h)
    assert out["jumps"] == 2 and out["jump_sites"] == 2
    by = {}
    for i, amp in zip(d.addr, d.amp):
        by.setdefault(int(i), []).append(abs(amp) ** 2)
    assert sorted(by) == list(range(1 << (n - 1), 1 << n))
    for i, w in by.items():
        assert len(w) == 2, (i, len(w))
        w = sorted(w, reverse=True)
        assert abs(w[1] / w[0] - a2 ** _window(n, 1, s_stop)) < 1e-12, (i, w)


def test_data_qubit_positions_are_shared_by_the_configurations():
    """After the router jump, with every data qubit in the tree, the excited
    sites of a branch's 2^k configurations are one address part plus exactly
    the subsets of k data-slot sites (the data qubits' positions, the same in
    every configuration): the masks of the product form."""
    n, k, gamma, s_stop = 4, 3, 0.1, 15
    assert max(cf.tau_in(n, t) for t in range(k)) <= s_stop < min(cf.tau_out(n, t) for t in range(k))
    p = W.data_loading(W.QUBIT, n, k, seed=7)
    h = core.History(cand_slice=[5], cand_site=[0], aux_u={5: 0.999}, final_u=0.5, stop_slice=s_stop)
    _, d = core.run_one(p, 7, 0, gamma, hist=h)
    by = {}
    for i, b, c in zip(d.addr, d.bus, d.configs):
        by.setdefault(int(i), []).append((int(b), frozenset(c)))
    assert len(by) == 1 << (n - 1)
    positions = set()
    for i, comps in by.items():
        assert len(comps) == 1 << k and all(b == 0 for b, _ in comps)     # every data qubit is out of the bus
        sets = [c for _, c in comps]
        common = frozenset.intersection(*sets)
        extras = [c - common for c in sets]
        sites = frozenset().union(*extras)
        assert len(sites) == k and all(site % 2 == 1 and lvl == 1 for site, lvl in sites)   # data slots
        subsets = {frozenset(x) for r in range(k + 1) for x in itertools.combinations(sites, r)}
        assert set(extras) == subsets, (i, extras)
        positions.add(sites)
    assert len(positions) > 1          # the positions depend on the branch's address bits
