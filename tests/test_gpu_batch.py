"""Mixed persistent launch: one graph-captured, work-stealing launch over
problems of different encodings, address widths n and data widths k.  Every
trajectory's result must be bitwise the one its problem's own launch gives in
the same launch variant, and a sample of each problem must match the CPU
oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import core

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _problems():
    # (problem, seed, first trajectory, damping rates)
    g6 = np.tile([1e-4, 1e-3, 1e-2], 1000)
    g12 = W.gamma_batches(600, 100, 1e-5, 1e-2, seed=4001)
    return [
        (W.data_loading(W.QUTRIT, 10, 1, seed=3001), 3001, 0, np.full(2000, 1e-3)),
        (W.data_loading(W.QUBIT, 6, 1, seed=2001), 2001, 500, g6),
        (W.data_loading(W.QUBIT, 12, 4, seed=4001), 4001, 77, g12),
        (W.random_columns(W.QUBIT, 4, 3, D=11, seed=9), 9, 0, np.full(500, 2e-2)),
    ]


def _setup(threads):
    from paper_2609_34935_b300 import QramSim
    sims, gams, outs, t0s, probs = [], [], [], [], []
    for p, seed, t0, g in _problems():
        sim = QramSim(p, seed=seed, device=0)
        sim.set_gamma_bound(float(g.max()))
        sims.append(sim)
        gams.append(torch.tensor(g, dtype=torch.float64, device="cuda:0"))
        outs.append(torch.full((len(g), 48), 0xCD, dtype=torch.uint8, device="cuda:0"))
        t0s.append(t0)
        probs.append((p, seed, t0, g))
    return sims, gams, outs, t0s, probs


@pytest.mark.parametrize("mode,threads", [("pruned", 256), ("pruned", 512), ("full", 256)])
def test_mixed_launch_equals_each_problem_alone(mode, threads):
    from paper_2609_34935_b300 import QramBatch, QramSim
    sims, gams, outs, t0s, probs = _setup(threads)
    batch = QramBatch(sims, mode, t0s, gams, outs, threads=threads)
    assert batch.grid >= 1
    for rep in range(2):                               # the graph replays: same results
        for o in outs:
            o.fill_(0xCD)
        batch()
        torch.cuda.synchronize()
        for sim, g, o, t0 in zip(sims, gams, outs, t0s):
            assert sim.variant == threads
            alone = sim.run(mode, t0, g).cpu().numpy()
            assert np.array_equal(o.cpu().numpy(), alone)
    for (p, seed, t0, g), o in zip(probs, outs):
        got = QramSim.results(o)
        assert np.all(got["status"] == 0)
        sel = np.arange(0, len(g), max(1, len(g) // 40))
        ref = np.concatenate([core.run(p, seed, t0 + int(t), g[t:t + 1]) for t in sel])
        for f in ("bad", "ref", "ncand", "jumps", "first_jump_slice", "q_ground"):
            assert np.array_equal(got[f][sel].astype(np.int64), ref[f].astype(np.int64)), f
        for f in ("fidelity", "fidelity_unsampled", "p_ground"):
            assert np.max(np.abs(got[f][sel] - ref[f])) < TOL, f
    batch.close()
    for sim in sims:
        sim.close()


def test_mixed_launch_preconditions():
    from paper_2609_34935_b300 import QramBatch, QramError, QramSim
    p = W.data_loading(W.QUBIT, 5, 2, seed=1)
    sim = QramSim(p, seed=1, device=0)
    g = torch.full((10,), 1e-3, dtype=torch.float64, device="cuda:0")
    o = torch.empty((10, 48), dtype=torch.uint8, device="cuda:0")
    with pytest.raises(QramError) as e:                # no damping-rate bound
        QramBatch([sim], "pruned", [0], [g], [o])
    assert e.value.code == 7
    sim.set_gamma_bound(1e-3)
    sim.set_depolarizing(1e-3)
    with pytest.raises(QramError) as e:                # depolarizing faults are not batched
        QramBatch([sim], "pruned", [0], [g], [o])
    assert e.value.code == 1
    sim.set_depolarizing(0.0)
    b = QramBatch([sim], "pruned", [0], [g], [o])
    b()
    torch.cuda.synchronize()
    assert np.array_equal(o.cpu().numpy(), sim.run_pruned(0, g).cpu().numpy())
    b.close()
    sim.close()
