"""Serving loop (continuous batching) through the C ABI: requests of mixed
encoding, n, k, gamma and trajectory count, admitted by device-memory
budget, must return exactly the results they give alone; host-side failures
(malformed, oversized, cancelled requests) are reported per request."""
import ctypes as C
import time

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _server(budget=8 << 30, max_active=4):
    from paper_2609_34935_b300 import QramServer
    return QramServer(budget, device=0, max_active=max_active)


def _requests(seed=5001, count=12):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        enc = int(rng.integers(0, 2))
        n = int(rng.integers(4, 9))
        k = int(rng.integers(1, min(n, 4) + 1))
        gamma = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-2))))
        nt = int(np.exp(rng.uniform(np.log(50), np.log(400))))
        p = W.data_loading(enc, n, k, seed=seed * 1000 + i)
        reqs.append((p, seed * 1000 + i, 7 * i, np.full(nt, gamma), 0 if i % 3 else 1))
    return reqs


def _alone(p, seed, traj0, g, mode):
    from paper_2609_34935_b300 import QramSim
    sim = QramSim(p, seed=seed, device=0)
    r = QramSim.results(sim.run("pruned" if mode == 0 else "full", traj0, torch.tensor(g, device="cuda:0")))
    sim.close()
    return r


def test_mix_equals_alone():
    srv = _server()
    reqs = _requests()
    ids = [srv.submit(p, seed, traj0, g, mode) for p, seed, traj0, g, mode in reqs]
    assert srv.drain(300.0)
    comps = {c["id"]: c for c in srv.poll()}
    assert set(comps) == set(ids)
    overlap = 0
    for rid, (p, seed, traj0, g, mode) in zip(ids, reqs):
        c = comps[rid]
        assert c["status"] == 0
        got = srv.results(rid, len(g))
        ref = _alone(p, seed, traj0, g, mode)
        assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))          # bitwise the same
        assert abs(c["mean_fidelity"] - ref["fidelity"].mean()) < 1e-12
        assert c["t_submit"] <= c["t_admit"] <= c["t_finish"]
    # requests ran concurrently: some admission happened before an earlier request finished
    fin = sorted((comps[i]["t_admit"], comps[i]["t_finish"]) for i in ids)
    overlap = sum(1 for a, b in zip(fin, fin[1:]) if b[0] < a[1])
    assert overlap > 0
    srv.close()


def test_admission_by_memory_budget():
    """A budget that fits one request at a time still completes all of them
    (queued requests are admitted as memory frees up)."""
    from paper_2609_34935_b300 import QramServer
    reqs = [(W.data_loading(W.QUBIT, 7, 2, seed=70 + i), 70 + i, 0, np.full(300, 2e-3), 0) for i in range(4)]
    srv = QramServer(1 << 40, device=0, max_active=4)
    need = max(srv.estimate(r[0], len(r[3])) for r in reqs)
    srv.close()
    srv = QramServer(int(need * 1.2), device=0, max_active=4)
    ids = [srv.submit(*r) for r in reqs]
    assert srv.drain(300.0)
    comps = srv.poll()
    assert sorted(c["id"] for c in comps) == sorted(ids)
    assert all(c["status"] == 0 for c in comps)
    iv = sorted((c["t_admit"], c["t_finish"]) for c in comps)
    assert all(b[0] >= a[1] - 1e-3 for a, b in zip(iv, iv[1:]))      # never two at once
    srv.close()


def test_rejections_and_cancel():
    from paper_2609_34935_b300 import QramError
    srv = _server(budget=64 << 20)
    p = W.data_loading(W.QUBIT, 5, 2, seed=1)
    with pytest.raises(QramError) as e:                     # gamma outside [0, 1)
        srv.submit(p, 1, 0, np.array([0.5, 1.0]), 0)
    assert e.value.code == 1
    q = W.data_loading(W.QUBIT, 5, 2, seed=1)
    q.addr = q.addr.copy()
    q.addr[1] = q.addr[0]                                   # duplicate address
    with pytest.raises(QramError) as e:
        srv.submit(q, 1, 0, np.array([0.01]), 0)
    assert e.value.code == 1
    big = W.data_loading(W.QUBIT, 14, 4, seed=1)            # larger than the 64 MiB budget
    with pytest.raises(QramError) as e:
        srv.submit(big, 1, 0, np.full(10, 1e-3), 0)
    assert e.value.code == 2
    # cancel: a long request queued behind another; cancel the queued one
    srv2 = _server(budget=8 << 30, max_active=1)
    a = srv2.submit(W.data_loading(W.QUBIT, 8, 3, seed=2), 2, 0, np.full(3000, 1e-3), 0)
    b = srv2.submit(W.data_loading(W.QUBIT, 8, 3, seed=3), 3, 0, np.full(3000, 1e-3), 0)
    srv2.cancel(b)
    assert srv2.drain(300.0)
    st = {c["id"]: c["status"] for c in srv2.poll()}
    assert st[a] == 0 and st[b] == 7
    srv2.close()
    srv.close()
