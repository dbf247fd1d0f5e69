"""Brute-force density-matrix simulation of the whole loading circuit
(App. C, "Cross-check against an independent circuit-level simulation").

Test infrastructure only.  The register is unfolded gate by gate: n address
qubits, k bus qubits and, per routing node v, a router a_v and a data slot
d_v (qubits, or qutrits {W, L, R} for the qutrit encoding).  Every slice
applies its gates as a permutation (with signs) of basis states, then the
amplitude damping channel of Eq. (5) / Eq. (6) on every tree site with the
fixed Kraus matrices, no sampling.  Feasible for n <= 2 (qubit) and n = 1
(qutrit).  Written independently of ``qram_oracle.c``: the gate definitions
below are restated from App. C, not shared.
"""
from __future__ import annotations

import math

import numpy as np


def _events(n: int, k: int):
    """Gate list per slice of the time-sliced schedule (Sec. II.A)."""
    T = 6 * n + 2 * k
    ev = {s: [] for s in range(1, T)}

    def add(s, g):
        if g not in ev[s]:
            ev[s].append(g)
    for l in range(n):
        add(2 * l + 1, ("copy", l))
        for m in range(1, l + 1):
            add(2 * l + 1 + m, ("cswap", m - 1))
        add(3 * l + 2, ("iswap", l))
        add(T - 3 * l - 2, ("iswap", l))
        for m in range(1, l + 1):
            add(T - 2 * l - 1 - m, ("cswap", m - 1))
        add(T - 2 * l - 1, ("copy", l))
    for t in range(k):
        add(2 * n + 2 * t + 1, ("bus", t))
        for m in range(1, n):
            add(2 * n + 2 * t + 1 + m, ("cswap", m - 1))
        add(3 * n + 2 * t + 1, ("fetch", t))
        for m in range(1, n):
            add(3 * n + 2 * t + 1 + m, ("cswap", n - 1 - m))
        add(4 * n + 2 * t + 1, ("bus", t))
    return T, ev


def _weyl(d: int):
    """Non-identity Pauli (d = 2: X, Z, Y) or Weyl operators X^a Z^b (d = 3)."""
    X = np.roll(np.eye(d, dtype=np.complex128), 1, axis=0)          # |j> -> |j+1 mod d>
    w = np.exp(2j * math.pi / d)
    Z = np.diag([w ** j for j in range(d)])
    ops = []
    for a_ in range(d):
        for b_ in range(d):
            if a_ or b_:
                ops.append(np.linalg.matrix_power(X, a_) @ np.linalg.matrix_power(Z, b_))
    return ops


def simulate(encoding: int, n: int, k: int, memory, gamma: float, addr=None, bus=None, amp=None,
             eps: float = 0.0, depol_first: bool = True, channel: str = "damping"):
    """Returns (F_rho, trace, marginal distribution over (address, bus)).

    channel: "damping" (Eqs. (5)-(6)); "dephasing": the phase-damping
    channel with the same no-jump operator diag(1, a) (qutrit diag(1, a, a))
    and the jump sqrt(gamma)|1><1| (qutrit sqrt(gamma)|L><L|, sqrt(gamma)|R><R|);
    "heating": the no-jump operator diag(a, 1) (qutrit diag(a, 1, 1)) with the
    jump sqrt(gamma)|1><0| (qutrit sqrt(gamma/2)|L><W|, sqrt(gamma/2)|R><W|);
    the diagonal channels of the outlook (Sec. VII).

    eps: depolarizing channel of strength eps on every tree site after the
    gates of every slice (Sec. II.B): with probability eps one of the
    non-identity Paulis (qubits) or Weyl operators (qutrits), uniformly.
    depol_first: the depolarizing layer precedes the damping layer.
    Parity unpinned for eps > 0: App. C restricts the channel to the active
    positions of an undefined routing front, and Tab. IV's Pauli row is not
    reproduced with every site active; only trace preservation is checked."""
    nodes = (1 << n) - 1
    M = 2 * nodes
    base = 2 if encoding == 1 else 3
    radices = [base] * M + [2] * n + [2] * k      # tree sites, address (by layer), bus
    dim = int(np.prod(radices))
    strides = np.ones(len(radices), dtype=np.int64)
    for q in range(len(radices) - 2, -1, -1):
        strides[q] = strides[q + 1] * radices[q + 1]
    idx = np.arange(dim, dtype=np.int64)
    cfg0 = (idx[:, None] // strides[None, :]) % np.array(radices)[None, :]
    A0, B0 = M, M + n
    W, Lv, Rv = 0, 1, 2

    def encode(cfg):
        return (cfg * strides[None, :]).sum(axis=1)

    def gate(cfg, sign, g):
        cfg = cfg.copy()
        kind, p = g
        if kind == "copy":
            b = cfg[:, A0 + p]
            if encoding == 1:
                cfg[:, 1] ^= b
            else:
                tgt = np.where(b == 1, Rv, Lv)
                d0 = cfg[:, 1]
                cfg[:, 1] = np.where(d0 == W, tgt, np.where(d0 == tgt, W, d0))
        elif kind == "bus":
            q = B0 + p
            d0 = cfg[:, 1].copy()
            bb = cfg[:, q].copy()
            if encoding == 1:
                cfg[:, 1], cfg[:, q] = bb, d0
            else:
                mv = d0 != Lv
                cfg[:, 1] = np.where(mv, np.where(bb == 1, Rv, W), d0)
                cfg[:, q] = np.where(mv, (d0 == Rv).astype(cfg.dtype), bb)
        elif kind == "iswap":
            for v in range((1 << p) - 1, (2 << p) - 1):
                a, d = cfg[:, 2 * v].copy(), cfg[:, 2 * v + 1].copy()
                cfg[:, 2 * v], cfg[:, 2 * v + 1] = d, a
        elif kind == "cswap":
            for v in range((1 << p) - 1, (2 << p) - 1):
                r = cfg[:, 2 * v].copy()
                dv = cfg[:, 2 * v + 1].copy()
                dl = cfg[:, 2 * (2 * v + 1) + 1].copy()
                dr = cfg[:, 2 * (2 * v + 2) + 1].copy()
                if encoding == 1:
                    go_l, go_r = r == 0, r == 1
                else:
                    go_l, go_r = r == Lv, r == Rv
                cfg[:, 2 * v + 1] = np.where(go_l, dl, np.where(go_r, dr, dv))
                cfg[:, 2 * (2 * v + 1) + 1] = np.where(go_l, dv, dl)
                cfg[:, 2 * (2 * v + 2) + 1] = np.where(go_r, dv, dr)
        elif kind == "fetch":
            off = (1 << (n - 1)) - 1
            for v in range(off, nodes):
                r = cfg[:, 2 * v]
                for rv, cellbit in (((0, Lv)[encoding == 0], 0), ((1, Rv)[encoding == 0], 1)):
                    cell = 2 * (v - off) + cellbit
                    if not (int(memory[cell]) >> p) & 1:
                        continue
                    sel = r == rv
                    if encoding == 1:
                        sign = np.where(sel & (cfg[:, 2 * v + 1] == 1), -sign, sign)
                    else:
                        d = cfg[:, 2 * v + 1]
                        cfg[:, 2 * v + 1] = np.where(sel, np.where(d == W, Rv, np.where(d == Rv, W, d)), d)
        return cfg, sign

    T, ev = _events(n, k)
    # input state
    if addr is None:
        addr = list(range(1 << n))
        bus = [0] * (1 << n)
        amp = [2.0 ** (-n / 2)] * (1 << n)

    def basis(i, j):
        cfg = np.zeros(len(radices), dtype=np.int64)
        for l in range(n):
            cfg[A0 + l] = (i >> (n - 1 - l)) & 1
        for t in range(k):
            cfg[B0 + t] = (j >> t) & 1
        return int((cfg * strides).sum())

    psi = np.zeros(dim, dtype=np.complex128)
    psi_id = np.zeros(dim, dtype=np.complex128)
    for i, j, c in zip(addr, bus, amp):
        psi[basis(int(i), int(j))] += c
        psi_id[basis(int(i), int(j) ^ int(memory[int(i)]))] += c
    rho = np.outer(psi, psi.conj())
    a = math.sqrt(1.0 - gamma)
    sq = math.sqrt(gamma)

    def on_axis(rho, q, op):
        """rho -> (op on slot q) rho (op on slot q)^dagger"""
        shp = radices + radices
        r = rho.reshape(shp)
        r = np.moveaxis(np.tensordot(op, r, axes=([1], [q])), 0, q)
        qq = len(radices) + q
        r = np.moveaxis(np.tensordot(op.conj(), r, axes=([1], [qq])), 0, qq)
        return r.reshape(dim, dim)

    H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2)
    if channel not in ("damping", "dephasing", "heating"):
        raise ValueError(channel)
    if encoding == 1 and channel == "damping":
        kraus = [np.array([[1, 0], [0, a]], dtype=np.complex128),
                 np.array([[0, sq], [0, 0]], dtype=np.complex128)]
    elif encoding == 1 and channel == "heating":
        kraus = [np.diag([a, 1]).astype(np.complex128), np.array([[0, 0], [sq, 0]], dtype=np.complex128)]
    elif encoding == 1:
        kraus = [np.diag([1, a]).astype(np.complex128), np.diag([0, sq]).astype(np.complex128)]
    elif channel == "heating":
        h = math.sqrt(gamma / 2.0)
        kraus = [np.diag([a, 1, 1]).astype(np.complex128),
                 np.array([[0, 0, 0], [h, 0, 0], [0, 0, 0]], dtype=np.complex128),
                 np.array([[0, 0, 0], [0, 0, 0], [h, 0, 0]], dtype=np.complex128)]
    elif channel == "damping":
        kraus = [np.diag([1, a, a]).astype(np.complex128),
                 np.array([[0, sq, 0], [0, 0, 0], [0, 0, 0]], dtype=np.complex128),
                 np.array([[0, 0, sq], [0, 0, 0], [0, 0, 0]], dtype=np.complex128)]
    else:
        kraus = [np.diag([1, a, a]).astype(np.complex128), np.diag([0, sq, 0]).astype(np.complex128),
                 np.diag([0, 0, sq]).astype(np.complex128)]
    weyl = _weyl(base) if eps > 0 else []

    def depolarize(rho):
        for q in range(M):
            acc = (1.0 - eps) * rho
            for Wop in weyl:
                acc += (eps / len(weyl)) * on_axis(rho, q, Wop)
            rho = acc
        return rho

    def damp(rho):
        if gamma == 0.0:
            return rho
        for q in range(M):
            acc = np.zeros_like(rho)
            for K in kraus:
                acc += on_axis(rho, q, K)
            rho = acc
        return rho

    for s in range(1, T):
        if encoding == 1 and s == 2 * n + 1:
            for t in range(k):
                rho = on_axis(rho, B0 + t, H)
        cfg, sign = cfg0, np.ones(dim)
        for g in ev[s]:
            cfg, sign = gate(cfg, sign, g)
        P = encode(cfg)
        new = np.zeros_like(rho)
        new[np.ix_(P, P)] = (sign[:, None] * sign[None, :]) * rho
        rho = new
        if encoding == 1 and s == 4 * n + 2 * k - 1:
            for t in range(k):
                rho = on_axis(rho, B0 + t, H)
        if eps > 0 and depol_first:
            rho = depolarize(rho)
        rho = damp(rho)
        if eps > 0 and not depol_first:
            rho = depolarize(rho)
    F = float(np.real(psi_id.conj() @ rho @ psi_id))
    tr = float(np.real(np.trace(rho)))
    diag = np.real(np.diag(rho))
    marg = {}
    for x in np.nonzero(diag > 1e-300)[0]:
        c = cfg0[x]
        i = sum(int(c[A0 + l]) << (n - 1 - l) for l in range(n))
        j = sum(int(c[B0 + t]) << t for t in range(k))
        marg[(i, j)] = marg.get((i, j), 0.0) + float(diag[x])
    return F, tr, marg
