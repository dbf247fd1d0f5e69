"""Oracle pin for the joint damping sampler (Theorem 3, Eqs. (17)-(21)):
averaged over the candidate draw and the auxiliary draw, one layer of the
oracle reproduces the amplitude damping channel on every site exactly."""
import itertools
import math

import numpy as np
import pytest

from oracle import core


def _kraus(qubit, gamma, channel=core.DAMPING):
    a, s = math.sqrt(1 - gamma), math.sqrt(gamma)
    if channel == core.HEATING:                # diagonal no-jump operator on the ground level
        if qubit:
            return [np.diag([a, 1]), np.array([[0, 0], [s, 0]])]
        h = math.sqrt(gamma / 2)
        return [np.diag([a, 1, 1]), np.array([[0, 0, 0], [h, 0, 0], [0, 0, 0]]),
                np.array([[0, 0, 0], [0, 0, 0], [h, 0, 0]])]
    if channel == core.DEPHASING:              # phase damping: same no-jump operator, diagonal jumps
        if qubit:
            return [np.diag([1, a]), np.diag([0, s])]
        return [np.diag([1, a, a]), np.diag([0, s, 0]), np.diag([0, 0, s])]
    if qubit:
        return [np.array([[1, 0], [0, a]]), np.array([[0, s], [0, 0]])]
    return [np.diag([1, a, a]), np.array([[0, s, 0], [0, 0, 0], [0, 0, 0]]),
            np.array([[0, 0, s], [0, 0, 0], [0, 0, 0]])]


def _vec(comps, sites, base, nlab):
    """dense vector over (label, site levels)"""
    dim = nlab * base ** len(sites)
    v = np.zeros(dim, complex)
    for lab, (addr, bus, cfg, amp) in enumerate(comps):
        lv = dict(cfg)
        idx = addr
        for q in sites:
            idx = idx * base + lv.get(q, 0)
        v[idx] += amp
    return v


def _channel(rho, sites, base, nlab, kraus):
    nq = len(sites)
    shp = [nlab] + [base] * nq
    for pos in range(nq):
        r = rho.reshape(shp + shp)
        acc = 0
        for K in kraus:
            x = np.moveaxis(np.tensordot(K, r, axes=([1], [1 + pos])), 0, 1 + pos)
            x = np.moveaxis(np.tensordot(K.conj(), x, axes=([1], [len(shp) + 1 + pos])), 0, len(shp) + 1 + pos)
            acc = acc + x
        rho = acc.reshape(rho.shape)
    return rho


def _interval_mids(comps, cand):
    """u values at the middle of every interval of the canonical CDF: the
    masks J(x) = C n X(x), empty first, then sorted (site, level) lists."""
    W = sum(abs(c[3]) ** 2 for c in comps)
    groups = {}
    for addr, bus, cfg, amp in comps:
        J = tuple((q, l) for q, l in cfg if q in cand)
        groups[J] = groups.get(J, 0.0) + abs(amp) ** 2
    order = sorted(groups)                       # () sorts first; tuples lexicographic
    mids, cum = [], 0.0
    for J in order:
        w = groups[J]
        if w > 0:
            mids.append((J, (cum + w / 2) / W, w / W))
        cum += w
    return mids


@pytest.mark.parametrize("channel", [core.DAMPING, core.DEPHASING])
@pytest.mark.parametrize("qubit", [True, False])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_theorem3_single_layer(qubit, seed, channel):
    """Theorem 3 for amplitude damping, and its argument carried to the
    dephasing channel of the outlook: it needs only that K_J^dagger K_J is
    diagonal with the damping values, which holds for the phase-damping
    Kraus set with the same no-jump operator."""
    rng = np.random.default_rng(seed)
    base = 2 if qubit else 3
    sites = [1, 4, 5, 8]
    nlab = 3
    gamma = 0.27
    comps = []
    for lab in range(nlab):
        for _ in range(3):
            cfg = tuple((q, int(rng.integers(1, base))) for q in sites if rng.random() < 0.6)
            comps.append((lab, 0, cfg, complex(rng.normal(), rng.normal())))
    # merge duplicate keys
    d = {}
    for c in comps:
        d[(c[0], c[2])] = d.get((c[0], c[2]), 0) + c[3]
    comps = [(k[0], 0, k[1], v) for k, v in d.items()]
    nrm = math.sqrt(sum(abs(c[3]) ** 2 for c in comps))
    comps = [(a, b, c, v / nrm) for a, b, c, v in comps]
    psi = _vec(comps, sites, base, nlab)
    rho_in = np.outer(psi, psi.conj())
    want = _channel(rho_in, sites, base, nlab, _kraus(qubit, gamma, channel))
    got = np.zeros_like(rho_in)
    for mask in itertools.product([0, 1], repeat=len(sites)):
        cand = [q for q, m in zip(sites, mask) if m]
        pc = gamma ** len(cand) * (1 - gamma) ** (len(sites) - len(cand))
        for J, u, pj in _interval_mids(comps, set(cand)):
            out, Jo = core.joint_layer(comps, cand, gamma, u, channel)
            assert Jo == J
            v = _vec(out, sites, base, nlab)
            assert np.linalg.norm(v) == pytest.approx(1.0, abs=1e-12)
            got += pc * pj * np.outer(v, v.conj())
    assert np.max(np.abs(got - want)) < 1e-13


def _interval_mids_heat(comps, cand, levels):
    """Heating: the masks are the candidate sites a component holds at the
    ground level, with the candidates' target levels."""
    W = sum(abs(c[3]) ** 2 for c in comps)
    groups = {}
    for addr, bus, cfg, amp in comps:
        lv = dict(cfg)
        J = tuple((q, levels[q]) for q in sorted(cand) if lv.get(q, 0) == 0)
        groups[J] = groups.get(J, 0.0) + abs(amp) ** 2
    mids, cum = [], 0.0
    for J in sorted(groups):
        w = groups[J]
        if w > 0:
            mids.append((J, (cum + w / 2) / W, w / W))
        cum += w
    return mids


@pytest.mark.parametrize("qubit", [True, False])
@pytest.mark.parametrize("seed", [0, 1])
def test_theorem3_single_layer_heating(qubit, seed):
    """The joint sampler with masks over the ground sites reproduces the
    heating channel (diagonal no-jump operator on the ground level, jumps to
    the excited levels; qutrit target level drawn per candidate) exactly,
    averaged over candidates, target levels and the auxiliary draw."""
    rng = np.random.default_rng(10 + seed)
    base = 2 if qubit else 3
    sites = [1, 4, 5]
    nlab = 3
    gamma = 0.31
    d = {}
    for lab in range(nlab):
        for _ in range(3):
            cfg = tuple((q, int(rng.integers(1, base))) for q in sites if rng.random() < 0.5)
            d[(lab, cfg)] = d.get((lab, cfg), 0) + complex(rng.normal(), rng.normal())
    comps = [(k[0], 0, k[1], v) for k, v in d.items()]
    nrm = math.sqrt(sum(abs(c[3]) ** 2 for c in comps))
    comps = [(a, b, c, v / nrm) for a, b, c, v in comps]
    psi = _vec(comps, sites, base, nlab)
    rho_in = np.outer(psi, psi.conj())
    want = _channel(rho_in, sites, base, nlab, _kraus(qubit, gamma, core.HEATING))
    got = np.zeros_like(rho_in)
    for mask in itertools.product([0, 1], repeat=len(sites)):
        cand = [q for q, m in zip(sites, mask) if m]
        pc = gamma ** len(cand) * (1 - gamma) ** (len(sites) - len(cand))
        for tl in itertools.product([1] if qubit else [1, 2], repeat=len(cand)):
            levels = dict(zip(cand, tl))
            pt = 1.0 if qubit else 0.5 ** len(cand)
            for J, u, pj in _interval_mids_heat(comps, set(cand), levels):
                out, Jo = core.joint_layer(comps, cand, gamma, u, core.HEATING, levels)
                assert Jo == J
                v = _vec(out, sites, base, nlab)
                assert np.linalg.norm(v) == pytest.approx(1.0, abs=1e-12)
                got += pc * pt * pj * np.outer(v, v.conj())
    assert np.max(np.abs(got - want)) < 1e-13
