"""Parity at the largest supported sizes: address width n = 14 (the tree of
16383 routers) and data width k = 8 (256 wall configurations per branch, every
word of a product-form record in use), both encodings, both modes, against the
oracle trajectory by trajectory (integer outputs bit-exact, floating point
within 1e-12), and final amplitudes for k = 8."""
import numpy as np
import pytest

import workloads as W
from oracle import core

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12

CASES = [
    (W.QUBIT, 14, 4, 40, 3e-3, 160),
    (W.QUTRIT, 14, 2, 40, 3e-3, 160),
    (W.QUBIT, 8, 8, 20, 1e-2, 100),
    (W.QUBIT, 14, 8, 12, 2e-3, 60),
    (W.QUTRIT, 14, 8, 12, 2e-3, 100),
]


@pytest.mark.parametrize("enc,n,k,D,gamma,ntraj", CASES)
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_largest_sizes_match_oracle(enc, n, k, D, gamma, ntraj, mode):
    from paper_2609_34935_b300 import QramSim
    seed = 5100 + 31 * n + k
    p = W.random_columns(enc, n, k, D=D, seed=seed)
    g = np.full(ntraj, gamma)
    ref = core.run(p, seed, 0, g)
    sim = QramSim(p, seed=seed, device=0)
    got = sim.results(sim.run(mode, 0, torch.tensor(g, device="cuda:0")))
    sim.close()
    assert np.all(got["status"] == 0)
    for f in ("bad", "ref", "ncand", "jumps", "first_jump_slice", "jump_sites", "q_ground"):
        assert np.array_equal(got[f].astype(np.int64), ref[f].astype(np.int64)), f
    for f in ("fidelity", "fidelity_unsampled", "p_ground"):
        assert np.max(np.abs(got[f] - ref[f])) < TOL, f
    assert np.sum(ref["jumps"] > 0) >= ntraj // 4


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


@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_largest_data_width_amplitudes(mode):
    from paper_2609_34935_b300 import QramSim
    n, k, gamma, seed = 8, 8, 1e-2, 5377
    p = W.random_columns(W.QUBIT, n, k, D=6, seed=seed)
    sim = QramSim(p, seed=seed, device=0)
    jumped = 0
    for traj in range(6):
        r, d = core.run_one(p, seed, traj, gamma, None, cap=1 << 18)
        jumped += int(r["jumps"]) > 0
        want = {}
        for a, b, cfg, amp in zip(d.addr, d.bus, d.configs, d.amp):
            key = (int(a), int(b), _hash_cfg(cfg))
            want[key] = want.get(key, 0) + amp
        ga, gb, gh, gz = sim.dump_state(mode, traj, gamma)
        got = {}
        for a, b, h, z in zip(ga, gb, gh, gz):
            key = (int(a), int(b), int(h))
            got[key] = got.get(key, 0) + z
        for key in set(want) | set(got):
            assert abs(want.get(key, 0) - got.get(key, 0)) < TOL, (traj, key)
    sim.close()
    assert jumped >= 2
