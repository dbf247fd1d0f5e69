"""The fidelity-scan input (Sec. VI, restricted to one bus column per
address): min(D, 2^n) distinct addresses, bus words below 2^k, equal weights
with unit norm, reproducible from the seed."""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("n,k,D", [(3, 3, 500), (9, 3, 500), (12, 3, 500), (5, 2, 7)])
def test_uniform_random_input(n, k, D):
    p = W.uniform_random_input(W.QUBIT, n, k, D, seed=11)
    Dn = min(D, 1 << n)
    assert p.D == Dn
    assert len(np.unique(p.addr)) == Dn and int(p.addr.max()) < (1 << n)
    assert int(p.bus.max()) < (1 << k)
    assert np.allclose(np.abs(p.amp), 1 / np.sqrt(Dn)) and abs(np.sum(np.abs(p.amp) ** 2) - 1) < 1e-12
    q = W.uniform_random_input(W.QUBIT, n, k, D, seed=11)
    assert np.array_equal(p.addr, q.addr) and np.array_equal(p.bus, q.bus)
    if Dn == 1 << n:
        assert np.array_equal(np.sort(p.addr), np.arange(1 << n))
