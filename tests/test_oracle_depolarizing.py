"""Oracle pins for the depolarizing faults (Sec. II.B, App. A): the sampled
events have the binomial rate and uniform operators, and the trajectory
average of the fidelity matches the density-matrix oracle (an independent
implementation applying the channel as fixed Kraus matrices) for qubits at
n = 2 and qutrits at n = 1, alone and mixed with damping.  Reading: every
tree site is active in every slice (see the S4b note of qram_oracle.c)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import core
from oracle import dm


def _mean_se(f):
    return float(f.mean()), float(f.std(ddof=1) / math.sqrt(len(f)))


def test_pauli_events_rate_and_types():
    n, k, eps = 4, 2, 0.01
    for enc, ntypes in ((W.QUBIT, 3), (W.QUTRIT, 8)):
        p = W.data_loading(enc, n, k, seed=3)
        tot, trials, counts = 0, 0, np.zeros(ntypes)
        for t in range(60):
            sl, st, ty = core.sample_paulis(p, 17, t, eps)
            assert np.all(np.diff(sl.astype(np.int64) * 100000 + st) > 0)     # (slice, site) order, distinct
            tot += len(sl)
            trials += 2 * ((1 << n) - 1) * (cf.slices(n, k) - 1)
            counts += np.bincount(ty, minlength=ntypes)
        assert abs(tot - trials * eps) < 5 * math.sqrt(trials * eps * (1 - eps))
        exp = counts.sum() / ntypes
        chi2 = float(((counts - exp) ** 2 / exp).sum())
        assert chi2 < 3 * ntypes + 20                      # loose: uniform operators
        sl2, st2, ty2 = core.sample_paulis(p, 17, 59, eps)
        assert np.array_equal(sl, sl2) and np.array_equal(ty, ty2)


@pytest.mark.parametrize("gamma,eps", [(0.0, 0.02), (0.02, 0.02)])
def test_qubit_depolarizing_matches_density_matrix(gamma, eps):
    """n = 2, k = 1, memory 0110, data-loading input (the Tab. IV circuit)."""
    p = W.data_loading(W.QUBIT, 2, 1, seed=1)
    p.memory = np.array([0, 1, 1, 0], np.uint8)
    want, tr, _ = dm.simulate(W.QUBIT, 2, 1, p.memory, gamma, eps=eps)
    assert abs(tr - 1.0) < 1e-12
    N = 20000
    r = core.run(p, 4242, 0, np.full(N, gamma), eps=eps)
    assert np.all(r["status"] == 0)
    m, se = _mean_se(r["fidelity"])
    assert abs(m - want) < 5 * se + 1e-3, (m, se, want)


@pytest.mark.parametrize("gamma,eps", [(0.0, 0.05), (0.05, 0.05)])
def test_qutrit_depolarizing_matches_density_matrix(gamma, eps):
    p = W.data_loading(W.QUTRIT, 1, 1, seed=2)
    want, tr, _ = dm.simulate(W.QUTRIT, 1, 1, p.memory, gamma, eps=eps)
    assert abs(tr - 1.0) < 1e-12
    N = 20000
    r = core.run(p, 777, 0, np.full(N, gamma), eps=eps)
    m, se = _mean_se(r["fidelity"])
    assert abs(m - want) < 5 * se + 1e-3, (m, se, want)


def test_depolarizing_marks_bad_and_eps_gamma_mode():
    """Every event marks bad(v); eps < 0 ties eps to each trajectory's gamma."""
    p = W.data_loading(W.QUBIT, 5, 2, seed=4)
    g = np.full(40, 0.01)
    a = core.run(p, 9, 0, g, eps=0.01)
    b = core.run(p, 9, 0, g, eps=-1.0)
    assert np.array_equal(a["fidelity"], b["fidelity"]) and np.array_equal(a["bad"], b["bad"])
    c = core.run(p, 9, 0, g, eps=0.0)
    assert np.all(a["bad"] >= c["bad"]) and np.any(a["bad"] > c["bad"])
