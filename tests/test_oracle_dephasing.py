"""Oracle pins for the other diagonal channels of the outlook (Sec. VII).
Dephasing is taken as phase damping with the no-jump operator of Eq. (5),
heating as the no-jump operator diag(a, 1, 1) on the ground level with jumps
to the excited levels: their single-layer exactness is pinned in
test_oracle_joint.py; here
the trajectory average of the fidelity matches the density-matrix oracle
applying the fixed Kraus matrices (qubit n = 2 with the Tab. IV memory,
qutrit n = 1), jump-free trajectories keep the closed-form fidelity of the
damping closed forms (the no-jump evolution is the same operator), and a
dephasing jump leaves the configuration of its survivors unchanged."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import core
from oracle import dm


def _mean_se(f):
    return float(f.mean()), float(f.std(ddof=1) / math.sqrt(len(f)))


@pytest.mark.parametrize("gamma", [0.05, 0.2])
def test_qubit_dephasing_matches_density_matrix(gamma):
    p = W.data_loading(W.QUBIT, 2, 1, seed=1)
    p.memory = np.array([0, 1, 1, 0], np.uint8)
    want, tr, _ = dm.simulate(W.QUBIT, 2, 1, p.memory, gamma, channel="dephasing")
    assert abs(tr - 1.0) < 1e-12
    dmp, _, _ = dm.simulate(W.QUBIT, 2, 1, p.memory, gamma)
    assert abs(want - dmp) > 1e-3                      # a different channel, not a relabelled one
    N = 20000
    r = core.run(p, 5150, 0, np.full(N, gamma), channel=core.DEPHASING)
    assert np.all(r["status"] == 0)
    m, se = _mean_se(r["fidelity"])
    assert abs(m - want) < 5 * se + 1e-3, (m, se, want)


@pytest.mark.parametrize("gamma", [0.05, 0.3])
def test_qutrit_dephasing_matches_density_matrix(gamma):
    p = W.data_loading(W.QUTRIT, 1, 1, seed=2)
    want, tr, _ = dm.simulate(W.QUTRIT, 1, 1, p.memory, gamma, channel="dephasing")
    assert abs(tr - 1.0) < 1e-12
    N = 20000
    r = core.run(p, 778, 0, np.full(N, gamma), channel=core.DEPHASING)
    m, se = _mean_se(r["fidelity"])
    assert abs(m - want) < 5 * se + 1e-3, (m, se, want)


def test_dephasing_no_jump_fidelity_is_the_damping_closed_form():
    """K0 is the same operator in both channels, so every jump-free
    trajectory has the closed-form no-jump fidelity of Theorems 1-2."""
    n, k, gamma = 5, 2, 2e-3
    p = W.data_loading(W.QUBIT, n, k, seed=12)
    r = core.run(p, 31, 0, np.full(400, gamma), channel=core.DEPHASING)
    nj = r["jumps"] == 0
    assert nj.sum() > 50 and (~nj).sum() > 10
    F0 = cf.no_jump_fidelity(W.QUBIT, n, k, gamma, p.addr, p.bus, p.amp, p.memory)
    assert np.max(np.abs(r["fidelity"][nj] - F0)) < 1e-13


def test_dephasing_jump_keeps_the_configuration():
    """A fixed history with one jump: under dephasing the survivors hold the
    jumped site still excited (a projection), under damping it is lowered."""
    n, k = 3, 1
    p = W.data_loading(W.QUBIT, n, k, seed=3)
    s, site = 4, 0                                   # the root router, excited on half the branches
    hist = core.History([s], [site], aux_u={s: 0.999999}, stop_slice=s)
    _, dd = core.run_one(p, 9, 0, 0.3, hist, channel=core.DEPHASING)
    _, da = core.run_one(p, 9, 0, 0.3, hist, channel=core.DAMPING)
    assert len(dd.configs) > 0 and all(any(q == site for q, _ in cfg) for cfg in dd.configs)
    assert len(da.configs) > 0 and all(all(q != site for q, _ in cfg) for cfg in da.configs)


@pytest.mark.parametrize("enc,n,gamma,seed", [(W.QUBIT, 2, 0.01, 61), (W.QUBIT, 2, 0.03, 62), (W.QUTRIT, 1, 0.02, 63),
                                               (W.QUTRIT, 1, 0.08, 64)])
def test_heating_matches_density_matrix(enc, n, gamma, seed):
    """Heating excites idle sites of every branch: the trajectory mean of the
    fidelity matches the density-matrix oracle (qubit n=2 with the Tab. IV
    memory, qutrit n=1)."""
    p = W.data_loading(enc, n, 1, seed=seed)
    if enc == W.QUBIT:
        p.memory = np.array([0, 1, 1, 0], np.uint8)
    want, tr, _ = dm.simulate(enc, n, 1, p.memory, gamma, channel="heating")
    assert abs(tr - 1.0) < 1e-12
    N = 20000
    r = core.run(p, 900 + seed, 0, np.full(N, gamma), channel=core.HEATING)
    assert np.all(r["status"] == 0)
    m, se = _mean_se(r["fidelity"])
    assert abs(m - want) < 5 * se + 1e-3, (m, se, want)
    assert want < 0.99                                   # the channel does act
