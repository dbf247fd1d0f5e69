"""Closed forms of the paper, written out directly (test infrastructure only).

Each function restates one formula; the tests compare the C oracle's explicit
evolution against them.  Address bit "t" of Eq. (14) is the bit routed at
tree layer t, i.e. bit n-1-t of the address (most significant bit at the
root, the leaf ordering of Eq. (7)).
"""
from __future__ import annotations

import math


def slices(n: int, k: int) -> int:
    """T = 6n + 2k (Sec. II.A)."""
    return 6 * n + 2 * k


def tau_in(n: int, i: int) -> int:
    """Eq. (3): CopyIn slice of data qubit i."""
    return 2 * n + 2 * i + 1


def tau_fetch(n: int, i: int) -> int:
    """Eq. (3): fetch slice of data qubit i."""
    return 3 * n + 2 * i + 1


def tau_out(n: int, i: int) -> int:
    """Eq. (3): CopyOut slice of data qubit i."""
    return 4 * n + 2 * i + 1


def routed_bit(i: int, n: int, t: int) -> int:
    """Address bit routed at layer t."""
    return (i >> (n - 1 - t)) & 1


def c_addr(i: int, n: int, k: int) -> int:
    """Eq. (14): address exposure count of the qubit encoding."""
    T = slices(n, k)
    return sum(T - 2 * (2 * t + 1) for t in range(n) if routed_bit(i, n, t))


def c_qutrit(i: int, j: int, d: int, n: int, k: int) -> int:
    """Exposure count c(i, j) of Prop. 1 under the qutrit reading: every
    address item is excited (L or R) over the same T-4t-2 layers as Eq. (14);
    a data slot is excited (R) while it carries a 1, for n layers before the
    fetch with the input bit and n layers after it with the output bit."""
    T = slices(n, k)
    addr = sum(T - 4 * t - 2 for t in range(n))
    ham = bin(j).count("1") + bin(j ^ d).count("1")
    return addr + n * ham


def alpha(a: float, d: int) -> float:
    """Lemma 1: alpha_d = (1 + a^d) / 2."""
    return (1.0 + a ** d) / 2.0


def beta(a: float, d: int) -> float:
    """Lemma 1: beta_d = (1 - a^d) / 2."""
    return (1.0 - a ** d) / 2.0


def hamming_amplitude(c: int, b_out: int, k: int, a: float, n: int) -> float:
    """Eq. (13): A(c) = alpha_2n^(k-w) beta_2n^w, w = Ham(c xor b_out)."""
    w = bin(c ^ b_out).count("1")
    return alpha(a, 2 * n) ** (k - w) * beta(a, 2 * n) ** w


def good_branch_qubit(i: int, j: int, d: int, n: int, k: int, gamma: float) -> dict:
    """Eq. (16): unnormalised no-jump end state of good branch (i, j),
    word -> amplitude (times the input amplitude)."""
    a = math.sqrt(1.0 - gamma)
    pre = a ** c_addr(i, n, k)
    b_out = j ^ d
    return {c: pre * hamming_amplitude(c, b_out, k, a, n) for c in range(1 << k)}


def good_branch_qutrit(i: int, j: int, d: int, n: int, k: int, gamma: float) -> dict:
    """Eq. (8): a^c(i,j) |j xor d_i>."""
    a = math.sqrt(1.0 - gamma)
    return {j ^ d: a ** c_qutrit(i, j, d, n, k)}


def no_jump_norm_per_qubit(a: float, n: int) -> float:
    """Sec. IV.E: alpha^2 + beta^2 = (1 + a^(4n)) / 2."""
    return (1.0 + a ** (4 * n)) / 2.0


def leakage(gamma: float, n: int) -> float:
    """Eq. (23): beta^2 / (alpha^2 + beta^2) with d = 2n (exact)."""
    a = math.sqrt(1.0 - gamma)
    al, be = alpha(a, 2 * n), beta(a, 2 * n)
    return be * be / (al * al + be * be)


def leakage_asymptote(gamma: float, n: int) -> float:
    """Eq. (23): leading term n^2 gamma^2 / 4."""
    return n * n * gamma * gamma / 4.0


def channel_error_split(gamma: float, n: int):
    """Eq. (24): (1-a^2n)/2 = (1-a^4n)/4 + (1-a^2n)^2/4, returned as (lhs, rhs)."""
    a = math.sqrt(1.0 - gamma)
    lhs = (1.0 - a ** (2 * n)) / 2.0
    rhs = (1.0 - a ** (4 * n)) / 4.0 + (1.0 - a ** (2 * n)) ** 2 / 4.0
    return lhs, rhs


def mark_sources_total(n: int) -> float:
    """Eq. (25): sum_v |bad(v)| / 2^n = n + (n-1)(n-2)/4."""
    return n + (n - 1) * (n - 2) / 4.0


def p_good(count_sources: int, gamma: float, n: int, k: int) -> float:
    """Probability that an address is good: every one of the 2 sites of each
    of its marking-source nodes stays a non-candidate in all T-1 slices
    (candidates are independent with probability gamma, Sec. IV.D)."""
    return (1.0 - gamma) ** (2 * (slices(n, k) - 1) * count_sources)


def no_jump_fidelity(encoding: int, n: int, k: int, gamma: float, addr, bus, amp, memory) -> float:
    """Fidelity of a trajectory in which no jump fires: every branch follows
    its closed form (Eq. (8) or Eq. (16)); F = |<psi_id|psi>|^2 / <psi|psi>."""
    a = math.sqrt(1.0 - gamma)
    ov = 0.0
    nrm = 0.0
    for i, j, c in zip(addr, bus, amp):
        w = abs(complex(c)) ** 2
        d = int(memory[int(i)])
        if encoding == 1:
            pre = a ** c_addr(int(i), n, k)
            ov += w * pre * alpha(a, 2 * n) ** k
            nrm += w * pre * pre * no_jump_norm_per_qubit(a, n) ** k
        else:
            e = a ** c_qutrit(int(i), int(j), d, n, k)
            ov += w * e
            nrm += w * e * e
    return ov * ov / nrm
