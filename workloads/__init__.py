"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the simulated method: it only draws the
classical memory, the input columns and the per-batch damping rates that a
query simulation takes as inputs.  Everything is generated with numpy's
PCG64 from an explicit seed, so both sides see identical inputs.

Workloads (paper Sec. VI: data-loading input of one branch per address with
zero bus input; memory with i.i.d. uniform bits):
  - ``data_loading(n, k, seed)``: D = 2^n columns, c_i = 2^{-n/2}, bus 0.
  - ``random_columns(n, k, D, seed)``: D distinct addresses, random bus
    words, random complex amplitudes (one column per address, Sec. IV.D).
  - ``uniform_random_input(n, k, D, seed)``: min(D, 2^n) distinct addresses
    with random bus words and equal weights (the fidelity-scan input).
  - ``gamma_batches(ntraj, batch, lo, hi, seed)``: a damping rate per batch
    of trajectories, log-uniform in [lo, hi].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

QUTRIT = 0
QUBIT = 1


@dataclass
class Problem:
    """One QRAM query problem: encoding, sizes, memory and input columns."""

    encoding: int
    n: int
    k: int
    memory: np.ndarray      # uint8[2^n], bit t of memory[i] is d_i^(t)
    addr: np.ndarray        # uint32[D], distinct
    bus: np.ndarray         # uint32[D]
    amp: np.ndarray         # complex128[D], sum |amp|^2 = 1

    @property
    def D(self) -> int:
        return int(self.addr.shape[0])


def memory_bits(n: int, k: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 1 << k, size=1 << n, dtype=np.uint8)


def data_loading(encoding: int, n: int, k: int, seed: int) -> Problem:
    D = 1 << n
    return Problem(encoding, n, k, memory_bits(n, k, seed),
                   np.arange(D, dtype=np.uint32), np.zeros(D, dtype=np.uint32),
                   np.full(D, 2.0 ** (-n / 2), dtype=np.complex128))


def random_columns(encoding: int, n: int, k: int, D: int, seed: int) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed + 0x9E37))
    addr = np.sort(rng.choice(1 << n, size=D, replace=False)).astype(np.uint32)
    rng.shuffle(addr)
    bus = rng.integers(0, 1 << k, size=D, dtype=np.uint32)
    amp = rng.normal(size=D) + 1j * rng.normal(size=D)
    amp /= np.sqrt(np.sum(np.abs(amp) ** 2))
    return Problem(encoding, n, k, memory_bits(n, k, seed), addr, bus, amp.astype(np.complex128))


def uniform_random_input(encoding: int, n: int, k: int, D: int, seed: int) -> Problem:
    """The scan input of Sec. VI restricted to one bus column per address:
    min(D, 2^n) distinct addresses drawn without replacement, a uniform random
    bus word each, equal weights (the paper draws D of the 2^(n+k)
    address-bus components; several columns per address are outside the
    input class of Sec. IV.D)."""
    rng = np.random.Generator(np.random.PCG64(seed + 0x2E5))
    Dn = min(D, 1 << n)
    addr = np.sort(rng.choice(1 << n, size=Dn, replace=False)).astype(np.uint32)
    bus = rng.integers(0, 1 << k, size=Dn, dtype=np.uint32)
    amp = np.full(Dn, 1.0 / np.sqrt(Dn), dtype=np.complex128)
    return Problem(encoding, n, k, memory_bits(n, k, seed), addr, bus, amp)


def gamma_batches(ntraj: int, batch: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 0x51))
    nb = (ntraj + batch - 1) // batch
    g = np.exp(rng.uniform(np.log(lo), np.log(hi), size=nb))
    return np.repeat(g, batch)[:ntraj].astype(np.float64)


def fixed_gamma(ntraj: int, gamma: float) -> np.ndarray:
    return np.full(ntraj, gamma, dtype=np.float64)
