"""Fidelity versus address size (Fig. 2; damping only, or with depolarizing
faults of the same strength).

For each (n, gamma) point: one simulator on the scan input (min(D, 2^n)
distinct addresses, random bus words, equal weights; Sec. VI restricted to
one bus column per address), ``ntraj`` pruned trajectories in one launch,
and the trajectory mean of the fidelity with its standard error from the
library's fixed-order reduction (qram_fidelity).  Every step runs in the
CUDA library; this module only chooses the points and collects the numbers.
"""
from __future__ import annotations

import numpy as np

import workloads as W


def fidelity_vs_n(encoding: int = W.QUBIT, ns=range(2, 11), gammas=(1e-5, 1e-4, 1e-3), k: int = 3,
                  D: int = 500, ntraj: int = 200, seed: int = 6001, device: int = 0, eps_equals_gamma: bool = False):
    """Returns one dict per (n, gamma): mean fidelity, its standard error, the
    bad-branch fraction, the mean number of fired jumps and the sampled
    ground fraction.  eps_equals_gamma adds depolarizing faults of the same
    strength (the setting of Fig. 2)."""
    import torch
    from . import QramSim
    rows = []
    for n in ns:
        if k > n:
            continue
        p = W.uniform_random_input(encoding, n, k, D, seed + 97 * n)
        sim = QramSim(p, seed=seed + n, device=device)
        if eps_equals_gamma:
            sim.set_depolarizing(0.0, eps_equals_gamma=True)
        for g in gammas:
            gam = torch.full((ntraj,), float(g), dtype=torch.float64, device=f"cuda:{device}")
            raw = sim.run_pruned(0, gam)
            mean, se = sim.fidelity(raw)
            r = QramSim.results(raw)
            if not np.all(r["status"] == 0):
                raise RuntimeError(f"scan point n={n} gamma={g}: status {np.unique(r['status'])}")
            rows.append({"n": n, "gamma": float(g), "eps": float(g) if eps_equals_gamma else 0.0, "D": p.D, "mean_fidelity": mean, "se": se,
                         "bad_fraction": float(r["bad"].mean() / p.D), "jumps": float(r["jumps"].mean()),
                         "ground_fraction": float(r["q_ground"].mean())})
        sim.close()
    return rows
