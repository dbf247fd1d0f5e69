"""GPU parity for the dephasing channel (the diagonal channel of the outlook,
Sec. VII; qram_set_channel): trajectories in both modes and final amplitudes
against the oracle's full evolution under the same channel, on the same
seeded inputs.  Integer outputs bit-exact, floating point within 1e-12."""
import numpy as np
import pytest

import workloads as W
from oracle import core

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _problem(enc, n, k, kind, seed):
    if kind == "load":
        return W.data_loading(enc, n, k, seed=seed)
    if kind == "dm":
        p = W.data_loading(enc, n, k, seed=seed)
        p.memory = np.array([0, 1, 1, 0], np.uint8)
        return p
    return W.random_columns(enc, n, k, D=max(1, (1 << n) - 5), seed=seed)


def _sim(p, seed):
    from paper_2609_34935_b300 import QramSim
    sim = QramSim(p, seed=seed, device=0)
    sim.set_channel("dephasing")
    return sim


CASES = [
    (W.QUBIT, 2, 1, 0.05, 400, "dm"),
    (W.QUTRIT, 3, 1, 5e-2, 400, "load"),
    (W.QUBIT, 5, 2, 2e-2, 300, "load"),
    (W.QUBIT, 6, 1, 1e-2, 1000, "load"),
    (W.QUTRIT, 4, 2, 4e-2, 300, "rand"),
    (W.QUBIT, 5, 4, 2e-2, 200, "rand"),
    (W.QUBIT, 8, 3, 3e-3, 300, "load"),
    (W.QUTRIT, 8, 1, 3e-3, 300, "load"),
]


@pytest.mark.parametrize("enc,n,k,gamma,ntraj,kind", CASES)
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_dephasing_trajectories_match_oracle(enc, n, k, gamma, ntraj, kind, mode):
    seed = 9300 + 11 * n + k
    p = _problem(enc, n, k, kind, seed)
    g = np.full(ntraj, gamma)
    ref = core.run(p, seed, 0, g, channel=core.DEPHASING)
    sim = _sim(p, seed)
    got = sim.results(sim.run(mode, 0, torch.tensor(g, device="cuda:0")))
    sim.close()
    assert np.all(got["status"] == 0)
    for f in ("bad", "ref", "ncand", "jumps", "first_jump_slice", "jump_sites", "q_ground"):
        assert np.array_equal(got[f].astype(np.int64), ref[f].astype(np.int64)), f
    for f in ("fidelity", "fidelity_unsampled", "p_ground"):
        assert np.max(np.abs(got[f] - ref[f])) < TOL, f
    assert np.sum(ref["jumps"] > 0) > 0
    # the channel changes the outcome: damping on the same histories differs somewhere
    dmp = core.run(p, seed, 0, g)
    assert np.any(np.abs(dmp["fidelity"] - ref["fidelity"]) > 1e-9)


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


@pytest.mark.parametrize("enc,n,k,gamma,kind", [(W.QUBIT, 4, 3, 6e-2, "load"), (W.QUTRIT, 4, 2, 4e-2, "rand"),
                                               (W.QUBIT, 6, 2, 3e-3, "load"), (W.QUBIT, 5, 2, 1e-2, "rand")])
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_dephasing_final_state_amplitudes(enc, n, k, gamma, kind, mode):
    seed = 9500 + n
    p = _problem(enc, n, k, kind, seed)
    sim = _sim(p, seed)
    jumped = 0
    for traj in range(10):
        r, d = core.run_one(p, seed, traj, gamma, None, cap=1 << 16, channel=core.DEPHASING)
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
    assert jumped > 0
    sim.close()


HEAT_CASES = [
    (W.QUBIT, 2, 1, 0.01, 400, "dm"),
    (W.QUTRIT, 1, 1, 0.02, 400, "load"),
    (W.QUTRIT, 3, 1, 5e-3, 300, "load"),
    (W.QUBIT, 4, 2, 3e-3, 300, "load"),
    (W.QUTRIT, 4, 2, 2e-3, 200, "rand"),
    (W.QUBIT, 5, 3, 1e-3, 200, "rand"),
]


@pytest.mark.parametrize("enc,n,k,gamma,ntraj,kind", HEAT_CASES)
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_heating_trajectories_match_oracle(enc, n, k, gamma, ntraj, kind, mode):
    """Heating (qram_set_channel "heating"): every branch explicit in both
    modes, masks over the ground sites with drawn target levels."""
    from paper_2609_34935_b300 import QramSim
    seed = 9700 + 13 * n + k
    p = _problem(enc, n, k, kind, seed)
    g = np.full(ntraj, gamma)
    ref = core.run(p, seed, 0, g, channel=core.HEATING)
    sim = QramSim(p, seed=seed, device=0)
    sim.set_channel("heating")
    got = sim.results(sim.run(mode, 0, torch.tensor(g, device="cuda:0")))
    sim.close()
    assert np.all(got["status"] == 0)
    for f in ("bad", "ref", "ncand", "jumps", "first_jump_slice", "jump_sites", "q_ground"):
        assert np.array_equal(got[f].astype(np.int64), ref[f].astype(np.int64)), f
    for f in ("fidelity", "fidelity_unsampled", "p_ground"):
        assert np.max(np.abs(got[f] - ref[f])) < TOL, f
    assert np.sum(ref["jumps"] > 0) > 0


@pytest.mark.parametrize("enc,n,k,gamma,kind", [(W.QUBIT, 3, 2, 1e-2, "load"), (W.QUTRIT, 3, 2, 1e-2, "rand")])
def test_heating_final_state_amplitudes(enc, n, k, gamma, kind):
    from paper_2609_34935_b300 import QramSim
    seed = 9900 + n
    p = _problem(enc, n, k, kind, seed)
    sim = QramSim(p, seed=seed, device=0)
    sim.set_channel("heating")
    jumped = 0
    for traj in range(10):
        r, d = core.run_one(p, seed, traj, gamma, None, cap=1 << 16, channel=core.HEATING)
        jumped += int(r["jumps"]) > 0
        want = {}
        for a, b, cfg, amp in zip(d.addr, d.bus, d.configs, d.amp):
            key = (int(a), int(b), _hash_cfg(cfg))
            want[key] = want.get(key, 0) + amp
        for mode in ("pruned", "full"):
            ga, gb, gh, gz = sim.dump_state(mode, traj, gamma)
            got = {}
            for a, b, h, z in zip(ga, gb, gh, gz):
                key = (int(a), int(b), int(h))
                got[key] = got.get(key, 0) + z
            for key in set(want) | set(got):
                assert abs(want.get(key, 0) - got.get(key, 0)) < TOL, (traj, mode, key)
    assert jumped > 0
    sim.close()


def test_heating_excludes_depolarizing():
    from paper_2609_34935_b300 import QramError, QramSim
    sim = QramSim(W.data_loading(W.QUBIT, 3, 1, seed=1), seed=1, device=0)
    sim.set_channel("heating")
    with pytest.raises(QramError):
        sim.set_depolarizing(1e-3)
    sim.set_channel("damping")
    sim.set_depolarizing(1e-3)
    with pytest.raises(QramError):
        sim.set_channel("heating")
    sim.close()
