"""Launch order.  A pruned or full launch with more trajectories than CTAs
hands its trajectories out longest first (a cost score per trajectory from
its regenerated damping candidates, a counting sort on the device, then work
stealing over that permutation); results must not depend on it.  Each launch is compared bitwise, record by record, with the same
trajectories run in chunks no larger than the grid (index order, no sort),
eagerly and as a replayed graph, with zero, invalid and repeated rates mixed
in.  Every record must be written exactly once (the output is pre-filled with
a pattern no result has), and a sample matches the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import core

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
CHUNK = 128          # below any grid: these launches keep index order


def _rates(nt, seed):
    rng = np.random.default_rng(seed)
    g = 10.0 ** rng.uniform(-5.0, np.log10(3e-2), nt)
    g[rng.integers(0, nt, 40)] = 0.0
    g[rng.integers(0, nt, 300)] = 1e-2              # many equal rates: one bucket
    g[rng.integers(0, nt, 5)] = -1.0                 # invalid: QRAM_E_ARG, sorted last
    return g


def _chunked(sim, mode, t0, g):
    out = torch.full((len(g), 48), 0xCD, dtype=torch.uint8, device="cuda:0")
    gt = torch.tensor(g, dtype=torch.float64, device="cuda:0")
    for a in range(0, len(g), CHUNK):
        sim.run(mode, t0 + a, gt[a:a + CHUNK], out[a:a + CHUNK])
    return out.cpu().numpy()


@pytest.mark.parametrize("enc,n,k,mode", [(W.QUBIT, 6, 2, "pruned"), (W.QUTRIT, 6, 1, "pruned"),
                                          (W.QUBIT, 5, 3, "full")])
def test_sorted_launch_equals_index_order(enc, n, k, mode):
    from paper_2609_34935_b300 import QramSim
    seed, t0, nt = 7100 + 10 * n + k, 12345, 3000
    p = W.data_loading(enc, n, k, seed=seed)
    g = _rates(nt, seed)
    sim = QramSim(p, seed=seed, device=0)
    sim.set_gamma_bound(3e-2)
    want = _chunked(sim, mode, t0, g)

    gt = torch.tensor(g, dtype=torch.float64, device="cuda:0")
    out = torch.full((nt, 48), 0xCD, dtype=torch.uint8, device="cuda:0")
    l0 = sim.launch_count
    sim.run(mode, t0, gt, out)
    assert sim.launch_count - l0 == 3                 # the scores, the sort, then the trajectories
    got = out.cpu().numpy()
    assert not np.any(np.all(got == 0xCD, axis=1))    # every record written
    assert np.array_equal(got, want)

    # the same launch as a graph (sort and memory nodes inside it), replayed twice
    t0d = torch.tensor([t0], dtype=torch.int64, device="cuda:0")
    out.fill_(0xCD)
    graph = sim.graph(mode, gt, out, t0d)
    for _ in range(2):
        out.fill_(0xCD)
        l0 = sim.launch_count
        graph()
        torch.cuda.synchronize()
        assert sim.launch_count - l0 == 3
        assert np.array_equal(out.cpu().numpy(), want)
    graph.close()

    res = QramSim.results(out)
    bad = g < 0
    assert np.all(res["status"][bad] != 0) and np.all(res["status"][~bad] == 0)
    sel = np.flatnonzero(~bad)[::97]
    ref = np.concatenate([core.run(p, seed, t0 + int(t), g[t:t + 1]) for t in sel])
    for f in ("bad", "ref", "ncand", "jumps", "first_jump_slice", "q_ground"):
        assert np.array_equal(res[f][sel].astype(np.int64), ref[f].astype(np.int64)), f
    for f in ("fidelity", "fidelity_unsampled", "p_ground"):
        assert np.max(np.abs(res[f][sel] - ref[f])) < TOL, f
    sim.close()


def test_small_launch_is_not_sorted():
    from paper_2609_34935_b300 import QramSim
    p = W.data_loading(W.QUBIT, 5, 2, seed=3)
    sim = QramSim(p, seed=3, device=0)
    sim.set_gamma_bound(1e-2)
    g = torch.full((CHUNK,), 1e-3, dtype=torch.float64, device="cuda:0")
    l0 = sim.launch_count
    sim.run_pruned(0, g)
    torch.cuda.synchronize()
    assert sim.launch_count - l0 == 1                 # no more trajectories than CTAs: index order
    sim.close()
