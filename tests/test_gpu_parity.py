"""GPU parity: the CUDA path through the C ABI against the CPU oracle, on the
same seeded inputs.  Integer outputs (candidates, the bad union, B, the
reference branch, jump records, the sampled tree outcome) must match
bit-exactly; floating-point outputs within 1e-12 absolute (the tolerance the
method's FP64 arithmetic allows: both sides carry ~1e-16 relative rounding
per operation over at most a few thousand operations)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import core

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _sim(p, seed):
    from paper_2609_34935_b300 import QramSim
    return QramSim(p, seed=seed, device=0)


def _cmp_results(got, ref, check_bad=True):
    assert np.all(got["status"] == 0), np.unique(got["status"])
    if check_bad:
        assert np.array_equal(got["bad"], ref["bad"])
        assert np.array_equal(got["ref"], ref["ref"])
    assert np.array_equal(got["ncand"], ref["ncand"])
    assert np.array_equal(got["jumps"], ref["jumps"])
    assert np.array_equal(got["first_jump_slice"], ref["first_jump_slice"])
    assert np.array_equal(got["jump_sites"], ref["jump_sites"])
    assert np.array_equal(got["q_ground"], ref["q_ground"])
    for f in ("fidelity", "fidelity_unsampled", "p_ground"):
        d = np.abs(got[f] - ref[f])
        assert np.max(d) < TOL, (f, np.max(d), int(np.argmax(d)))


CASES = [
    # encoding, n, k, gamma, ntraj, input
    (W.QUTRIT, 3, 1, 1e-3, 1000, "load"),        # 8 cells, qutrit, k=1
    (W.QUTRIT, 3, 1, 5e-2, 400, "load"),
    (W.QUBIT, 6, 1, 1e-4, 300, "load"),          # 64 cells, phase-kickback fetch
    (W.QUBIT, 6, 1, 1e-3, 300, "load"),
    (W.QUBIT, 6, 1, 1e-2, 200, "load"),
    (W.QUBIT, 4, 3, 6e-2, 300, "load"),          # several-element joint outcomes
    (W.QUTRIT, 5, 2, 3e-2, 300, "rand"),
    (W.QUBIT, 5, 4, 2e-2, 200, "rand"),          # complex amplitudes, random bus
    (W.QUBIT, 1, 1, 0.2, 300, "load"),
    (W.QUTRIT, 1, 1, 0.3, 300, "load"),
    (W.QUBIT, 2, 1, 0.05, 400, "dm"),            # the Tab. IV setting
]


def _problem(enc, n, k, kind, seed):
    if kind == "load":
        return W.data_loading(enc, n, k, seed=seed)
    if kind == "dm":
        p = W.data_loading(enc, n, k, seed=seed)
        p.memory = np.array([0, 1, 1, 0], np.uint8)
        return p
    return W.random_columns(enc, n, k, D=max(1, (1 << n) - 5), seed=seed)


@pytest.mark.parametrize("enc,n,k,gamma,ntraj,kind", CASES)
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_trajectories_match_oracle(enc, n, k, gamma, ntraj, kind, mode):
    seed = 1000 + 17 * n + k
    p = _problem(enc, n, k, kind, seed)
    g = np.full(ntraj, gamma)
    ref = core.run(p, seed, 0, g)
    sim = _sim(p, seed)
    got = sim.results(sim.run(mode, 0, torch.tensor(g, device="cuda:0")))
    _cmp_results(got, ref)
    if mode == "pruned":
        assert np.all(got["explicit_comps"] == (got["bad"] + (got["ref"] >= 0)) << (k if enc == W.QUBIT else 0))
    sim.close()


@pytest.mark.parametrize("enc,n,k,gamma", [(W.QUTRIT, 10, 1, 1e-3), (W.QUBIT, 12, 4, 1e-3), (W.QUBIT, 7, 3, 3e-3)])
def test_sample_faults_bit_exact(enc, n, k, gamma):
    seed = 3001 + n
    p = W.data_loading(enc, n, k, seed=seed)
    nt = 6
    sim = _sim(p, seed)
    out = sim.sample_faults(5, torch.full((nt,), gamma, dtype=torch.float64, device="cuda:0"), cap=1 << 13)
    for t in range(nt):
        sl, st, bad, B, ref = core.sample_faults(p, seed, 5 + t, gamma)
        nc = int(out["ncand"][t])
        assert nc == len(sl)
        packed = out["cand"][t, :nc].cpu().numpy().astype(np.uint32)
        assert np.array_equal(packed >> 16, sl.astype(np.uint32))
        assert np.array_equal(packed & 0xFFFF, st.astype(np.uint32))
        bits = out["bad_bits"][t].cpu().numpy().astype(np.uint32)
        gbad = np.array([(bits[a >> 5] >> (a & 31)) & 1 for a in range(1 << n)], np.uint8)
        assert np.array_equal(gbad, bad)
        assert int(out["bad"][t]) == B and int(out["ref"][t]) == ref
    sim.close()


@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_full_size_qubit_n12_k4_sampled(mode):
    """The n=12, k=4 workload in the launch configuration of the benchmark,
    on a sample of trajectories the oracle can afford, across the gamma
    decades of the log-uniform draw."""
    p = W.data_loading(W.QUBIT, 12, 4, seed=4001)
    g = np.array([1e-5, 3e-5, 1e-4, 4e-4, 1e-3])
    ref = core.run(p, 4001, 77, g)
    sim = _sim(p, 4001)
    got = sim.results(sim.run(mode, 77, torch.tensor(g, device="cuda:0")))
    _cmp_results(got, ref)
    sim.close()


def _hash_cfg(cfg):
    """FNV-1a 64 over (site << 2 | level) little-endian words (the dump's hash)."""
    if not cfg:
        return 0
    h = 1469598103934665603
    for q, lv in cfg:
        v = (q << 2) | lv
        for b in range(4):
            h ^= (v >> (8 * b)) & 0xFF
            h = (h * 1099511628211) & (2 ** 64 - 1)
    return h or 1


DUMP_CASES = [
    # encoding, n, k, gamma, input, both jump-free and jumped trajectories among the 12
    (W.QUBIT, 4, 3, 6e-2, "load", False), (W.QUTRIT, 4, 2, 4e-2, "rand", False),
    (W.QUBIT, 5, 2, 1e-2, "rand", True), (W.QUBIT, 3, 3, 0.0, "load", False),
    (W.QUBIT, 6, 2, 3e-3, "load", True),      # every address, equal weights: the product-form lazy epochs
    (W.QUBIT, 8, 2, 1e-3, "load", True),
    (W.QUBIT, 6, 3, 4e-3, "rand", True),      # unequal complex weights: FP64 lazy weights
    (W.QUTRIT, 6, 1, 3e-3, "load", True),     # integer exponent histograms
]


@pytest.mark.parametrize("enc,n,k,gamma,kind,mix", DUMP_CASES)
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_final_state_amplitudes(enc, n, k, gamma, kind, mix, mode):
    """Final amplitudes of every component, keyed by (address, bus word,
    tree configuration), against the oracle's full evolution at 1e-12.  In
    pruned mode the dump runs the lazy form that qram_run_pruned runs (the
    closed-form branch-epoch counter moves): a jump-free trajectory comes
    entirely from the closed forms, a jumped one from the configurations
    materialised at its first jump."""
    seed = 555 + n
    p = _problem(enc, n, k, kind, seed)
    sim = _sim(p, seed)
    sim.work_counters(reset=True)
    jumped = []
    for traj in range(12):
        r, d = core.run_one(p, seed, traj, gamma, None, cap=1 << 16)
        jumped.append(int(r["jumps"]) > 0)
        want = {}
        for a, b, cfg, amp in zip(d.addr, d.bus, d.configs, d.amp):
            want[(int(a), int(b), _hash_cfg(cfg))] = amp
        ga, gb, gh, gz = sim.dump_state(mode, traj, gamma)
        got = {}
        for a, b, h, z in zip(ga, gb, gh, gz):
            key = (int(a), int(b), int(h))
            got[key] = got.get(key, 0) + z
        for key in set(want) | set(got):
            assert abs(want.get(key, 0) - got.get(key, 0)) < TOL, (traj, key)
    w = sim.work_counters(reset=True)
    if mode == "pruned":
        assert w["branch_epochs"] > 0                 # the lazy form ran
    if mix:
        assert any(jumped) and not all(jumped)
    sim.close()


def test_fixed_history_annihilation():
    """A fired jump on the reference's path annihilates every predicted good
    group (Sec. VI.A); fixed histories exercise it independently of the FAULT
    stream."""
    n, k = 5, 2
    p = W.data_loading(W.QUBIT, n, k, seed=9)
    T = 6 * n + 2 * k
    seed = 4242
    hist = []
    # candidates on d_0 while address bits travel: jump fires with high probability
    for t in range(24):
        s = 1 + (t % (T - 2))
        hist.append([(s, 1), (min(T - 1, s + 3), 2 * ((t % 7) + 1))])
    cand, off = [], [0]
    refs = []
    for h in hist:
        h = sorted(h)
        cand += [(s << 16) | q for s, q in h]
        off.append(len(cand))
        refs.append(h)
    sim = _sim(p, seed)
    sim.set_fault_history(torch.tensor(np.array(cand, np.int64).astype(np.int32), device="cuda:0"),
                          torch.tensor(np.array(off, np.int32), device="cuda:0"))
    g = np.full(len(hist), 0.02)
    for mode in ("pruned", "full"):
        got = sim.results(sim.run(mode, 0, torch.tensor(g, device="cuda:0")))
        fired = 0
        for t, h in enumerate(refs):
            r, _ = core.run_one(p, seed, t, 0.02, core.History([s for s, _ in h], [q for _, q in h]), cap=1 << 12)
            assert got["status"][t] == 0
            assert got["jumps"][t] == r["jumps"] and got["first_jump_slice"][t] == r["first_jump_slice"]
            assert got["bad"][t] == r["bad"] and got["ref"][t] == r["ref"]
            assert abs(got["fidelity"][t] - r["fidelity"]) < TOL
            assert abs(got["fidelity_unsampled"][t] - r["fidelity_unsampled"]) < TOL
            fired += int(r["jumps"] > 0)
        assert fired > 3
    sim.set_fault_history()
    sim.close()


def test_no_jump_trajectories_closed_form():
    """Qubit n=6, k=1: every trajectory without a fired jump returns the
    closed-form no-jump fidelity (Theorems 1-2)."""
    p = W.data_loading(W.QUBIT, 6, 1, seed=2001)
    sim = _sim(p, 2001)
    for gamma in (1e-4, 1e-3, 1e-2):
        got = sim.results(sim.run_pruned(0, torch.full((10000,), gamma, dtype=torch.float64, device="cuda:0")))
        F0 = cf.no_jump_fidelity(W.QUBIT, 6, 1, gamma, p.addr, p.bus, p.amp, p.memory)
        nj = got[got["jumps"] == 0]
        assert len(nj) > 100
        assert np.max(np.abs(nj["fidelity"] - F0)) < TOL
    sim.close()


def test_deterministic_and_edge_cases():
    p = W.data_loading(W.QUBIT, 5, 2, seed=3)
    sim = _sim(p, 3)
    g = torch.full((500,), 2e-2, dtype=torch.float64, device="cuda:0")
    a = sim.run_pruned(10, g).cpu().numpy()
    b = sim.run_pruned(10, g).cpu().numpy()
    assert np.array_equal(a, b)
    # gamma = 0: nothing is bad, one explicit branch, F = 1
    r = sim.results(sim.run_pruned(0, torch.zeros(50, dtype=torch.float64, device="cuda:0")))
    assert np.all(r["bad"] == 0) and np.all(r["ref"] == 0) and np.all(r["explicit_comps"] == 4)
    assert np.max(np.abs(r["fidelity"] - 1.0)) < TOL
    # invalid rates are reported per trajectory
    r = sim.results(sim.run_pruned(0, torch.tensor([0.5, 1.0, -0.1], dtype=torch.float64, device="cuda:0")))
    assert list(r["status"]) == [0, 1, 1]
    sim.close()
    # one branch, n = k = 1
    q = W.Problem(W.QUBIT, 1, 1, np.array([1, 0], np.uint8), np.array([1], np.uint32), np.array([1], np.uint32),
                  np.array([1.0 + 0j]))
    ref = core.run(q, 8, 0, np.full(200, 0.1))
    sim = _sim(q, 8)
    _cmp_results(sim.results(sim.run_pruned(0, torch.full((200,), 0.1, dtype=torch.float64, device="cuda:0"))), ref)
    sim.close()


def test_fidelity_reduction():
    p = W.data_loading(W.QUTRIT, 3, 1, seed=1001)
    sim = _sim(p, 1001)
    raw = sim.run_pruned(0, torch.full((1000,), 1e-3 * 20, dtype=torch.float64, device="cuda:0"))
    m, s = sim.fidelity(raw)
    f = sim.results(raw)["fidelity"]
    assert abs(m - f.mean()) < 1e-13 and abs(s - f.std(ddof=1) / math.sqrt(len(f))) < 1e-12
    sim.close()


def test_cuda_graph_replay_matches_direct_launch():
    """One persistent batched launch captured in a CUDA graph and replayed for
    two batches (first trajectory index read from device memory) gives the
    same results as direct launches."""
    p = W.data_loading(W.QUBIT, 6, 2, seed=31)
    sim = _sim(p, 31)
    sim.set_gamma_bound(1e-2)
    g = torch.full((700,), 4e-3, dtype=torch.float64, device="cuda:0")
    out = torch.empty((700, 48), dtype=torch.uint8, device="cuda:0")
    t0 = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    graph = sim.graph("pruned", g, out, t0)
    for first in (0, 500):
        t0.fill_(first)
        graph()
        torch.cuda.synchronize()
        got = out.cpu().numpy().copy()
        ref = sim.run_pruned(first, g).cpu().numpy()
        assert np.array_equal(got, ref)
    graph.close()
    sim.close()


@pytest.mark.parametrize("threads", [128, 256, 512, 1024])
def test_launch_variants_match_oracle(threads):
    """Every launch variant (threads per CTA: the autotuner's three and the
    one-trajectory-per-SM latency variant) gives the oracle's results."""
    p = W.data_loading(W.QUBIT, 5, 3, seed=91)
    g = np.full(300, 2e-2)
    ref = core.run(p, 91, 0, g)
    sim = _sim(p, 91)
    sim.set_variant(threads)
    assert sim.variant == threads
    _cmp_results(sim.results(sim.run_pruned(0, torch.tensor(g, device="cuda:0"))), ref)
    sim.close()


def test_autotune_picks_a_variant_and_caches(tmp_path):
    import json
    p = W.data_loading(W.QUTRIT, 8, 1, seed=5)
    sim = _sim(p, 5)
    cache = str(tmp_path / "tune.json")
    best = sim.autotune("pruned", 3e-3, 1500, cache=cache)
    assert best in (128, 256, 512) and sim.variant == best
    table = json.load(open(cache))
    assert list(table.values())[0]["threads"] == best
    sim.set_variant(256)
    assert sim.autotune("pruned", 3e-3, 1500, cache=cache) == best      # served from the cache
    sim.close()


def test_work_counters_exact():
    """The kernel's work counters obey exact identities: every block of the
    fault stream ends with one terminating draw (draws = candidates + blocks);
    a full launch without damping evolves every component through T - 1
    slices; a pruned one without damping only folds the closed form once."""
    enc, n, k, ntraj = W.QUBIT, 6, 2, 200
    p = W.data_loading(enc, n, k, seed=77)
    sim = _sim(p, 77)
    T = cf.slices(n, k)
    nblk = math.ceil((T - 1) * 2 * ((1 << n) - 1) / 2048)
    sim.work_counters(reset=True)
    r = sim.results(sim.run_pruned(0, torch.full((ntraj,), 3e-3, dtype=torch.float64, device="cuda")))
    w = sim.work_counters(reset=True)
    assert w["draws"] == int(r["ncand"].sum()) + ntraj * nblk
    g0 = torch.zeros(ntraj, dtype=torch.float64, device="cuda")
    sim.results(sim.run_full(0, g0))
    w = sim.work_counters(reset=True)
    assert w["draws"] == 0
    # one merged component per branch through slices 1..2n (before the first
    # wall its 2^k configurations share the tree), one in product form from
    # 2n+1 to 4n+2k-1 (the data qubits follow the routers whatever their
    # values), then one binomial group per branch (every data qubit back in
    # the bus): three epochs of one component per branch
    assert w["comp_slices"] == ntraj * p.D * (T - 1)
    assert w["comp_epochs"] == ntraj * p.D * 3
    sim.results(sim.run_pruned(0, g0))
    w = sim.work_counters(reset=True)
    assert w["comp_slices"] == 0 and w["comp_epochs"] == 0
    assert w["branch_epochs"] == ntraj * p.D
    sim.close()


@pytest.mark.parametrize("n,gamma", [(3, 1e-3), (5, 3e-3), (6, 1e-2)])
def test_fidelity_scan_points_match_oracle(n, gamma):
    """Points of the fidelity-vs-n scan (scan input: distinct addresses,
    random bus words, equal weights): every trajectory against the oracle,
    and the scan's mean and standard error against the oracle's numbers."""
    from paper_2609_34935_b300.scan import fidelity_vs_n
    k, D, ntraj, seed = 3, 500, 200, 6001
    rows = fidelity_vs_n(W.QUBIT, [n], [gamma], k=k, D=D, ntraj=ntraj, seed=seed)
    assert len(rows) == 1
    p = W.uniform_random_input(W.QUBIT, n, k, D, seed + 97 * n)
    ref = core.run(p, seed + n, 0, np.full(ntraj, gamma))
    sim = _sim(p, seed + n)
    got = sim.results(sim.run_pruned(0, torch.full((ntraj,), gamma, dtype=torch.float64, device="cuda:0")))
    sim.close()
    _cmp_results(got, ref)
    f = ref["fidelity"]
    assert abs(rows[0]["mean_fidelity"] - f.mean()) < TOL
    assert abs(rows[0]["se"] - f.std(ddof=1) / math.sqrt(ntraj)) < 1e-8
    assert rows[0]["D"] == min(D, 1 << n)


@pytest.mark.parametrize("wmax", [0, 1])
def test_dump_low_weight_truncation(wmax):
    """The truncated dump keeps exactly the good-branch output words within
    Hamming distance w_max of the ideal word (and every explicit component),
    with the same amplitudes as the complete dump."""
    n, k, gamma = 5, 4, 4e-3
    p = W.data_loading(W.QUBIT, n, k, seed=91)
    sim = _sim(p, 91)
    seen_drop = False
    for traj in range(6):
        ga, gb, gh, gz = sim.dump_state("pruned", traj, gamma)
        ta, tb, th, tz = sim.dump_state("pruned", traj, gamma, w_max=wmax)
        full = {(int(a), int(b), int(h)): z for a, b, h, z in zip(ga, gb, gh, gz)}
        trunc = {(int(a), int(b), int(h)): z for a, b, h, z in zip(ta, tb, th, tz)}
        for key, z in full.items():
            a, b, h = key
            ideal = int(p.bus[list(p.addr).index(a)]) ^ int(p.memory[a])
            keep = h != 0 or bin(b ^ ideal).count("1") <= wmax or key in trunc
            if not keep:
                seen_drop = True
                continue
            assert key in trunc and abs(trunc[key] - z) < TOL
        assert set(trunc) <= set(full)
    sim.dump_state("pruned", 0, gamma, w_max=-1)
    assert seen_drop
    sim.close()


DEPOL_CASES = [
    # encoding, n, k, gamma, eps, ntraj, input
    (W.QUBIT, 2, 1, 0.0, 0.02, 400, "dm"),        # the Tab. IV circuit, Pauli only
    (W.QUBIT, 2, 1, 0.02, 0.02, 400, "dm"),       # mixed
    (W.QUBIT, 5, 3, 2e-3, 2e-3, 200, "load"),
    (W.QUBIT, 6, 2, 1e-3, -1.0, 200, "rand"),     # eps = gamma per trajectory
    (W.QUTRIT, 1, 1, 0.05, 0.05, 400, "load"),
    (W.QUTRIT, 4, 2, 4e-3, 4e-3, 200, "rand"),
]


@pytest.mark.parametrize("enc,n,k,gamma,eps,ntraj,kind", DEPOL_CASES)
@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_depolarizing_trajectories_match_oracle(enc, n, k, gamma, eps, ntraj, kind, mode):
    seed = 7000 + 13 * n + k
    p = _problem(enc, n, k, kind, seed)
    g = np.full(ntraj, gamma)
    ref = core.run(p, seed, 0, g, eps=eps)
    sim = _sim(p, seed)
    sim.set_depolarizing(max(eps, 0.0), eps_equals_gamma=eps < 0)
    got = sim.results(sim.run(mode, 0, torch.tensor(g, device="cuda:0")))
    _cmp_results(got, ref)
    sim.close()


@pytest.mark.parametrize("enc,n,k,gamma,eps", [(W.QUBIT, 3, 2, 0.03, 0.03), (W.QUTRIT, 3, 1, 0.02, 0.03)])
def test_depolarizing_final_state_amplitudes(enc, n, k, gamma, eps):
    seed = 8100 + n
    p = _problem(enc, n, k, "rand", seed)
    sim = _sim(p, seed)
    sim.set_depolarizing(eps)
    for traj in range(10):
        _, d = core.run_one(p, seed, traj, gamma, None, cap=1 << 14, eps=eps)
        want = {}
        for a, b, cfg, amp in zip(d.addr, d.bus, d.configs, d.amp):
            key = (int(a), int(b), _hash_cfg(cfg))
            want[key] = want.get(key, 0) + amp
        ga, gb, gh, gz = sim.dump_state("pruned", traj, gamma)
        got = {}
        for a, b, h, z in zip(ga, gb, gh, gz):
            key = (int(a), int(b), int(h))
            got[key] = got.get(key, 0) + z
        for key in set(want) | set(got):
            assert abs(want.get(key, 0) - got.get(key, 0)) < TOL, (traj, key)
    sim.close()


@pytest.mark.parametrize("mode", ["pruned", "full"])
def test_merged_components_before_the_first_wall(mode):
    """Jumps before the first Hadamard wall (slices <= 2n), while one merged
    component per branch stands for its 2^k wall configurations, then
    candidates in the data phase after the expansion: fixed histories
    against the oracle, trajectory by trajectory and amplitude by
    amplitude."""
    n, k = 6, 3
    p = W.random_columns(W.QUBIT, n, k, D=50, seed=17)
    T = 6 * n + 2 * k
    seed = 2718
    rng = np.random.default_rng(5)
    hists = []
    for t in range(40):
        early = sorted({(int(rng.integers(2, 2 * n + 1)), int(rng.integers(0, 2 * (2 ** n - 1))) % 8)
                        for _ in range(3)})
        late = sorted({(int(rng.integers(2 * n + 1, T)), int(rng.integers(0, 2 * (2 ** n - 1))))
                       for _ in range(6)})
        hists.append(sorted(set(early + late)))
    cand, off = [], [0]
    for h in hists:
        cand += [(s << 16) | q for s, q in h]
        off.append(len(cand))
    sim = _sim(p, seed)
    sim.set_fault_history(torch.tensor(np.array(cand, np.int64).astype(np.int32), device="cuda:0"),
                          torch.tensor(np.array(off, np.int32), device="cuda:0"))
    g = np.full(len(hists), 0.02)
    got = sim.results(sim.run(mode, 0, torch.tensor(g, device="cuda:0")))
    early_jumps = 0
    for t, h in enumerate(hists):
        r, _ = core.run_one(p, seed, t, 0.02, core.History([s for s, _ in h], [q for _, q in h]), cap=1 << 14)
        assert got["status"][t] == 0
        for f in ("jumps", "first_jump_slice", "jump_sites", "q_ground", "bad", "ref"):
            assert int(got[f][t]) == int(r[f]), (t, f)
        for f in ("fidelity", "fidelity_unsampled", "p_ground"):
            assert abs(got[f][t] - r[f]) < TOL, (t, f)
        early_jumps += int(0 < r["first_jump_slice"] <= 2 * n)
    assert early_jumps >= 3
    sim.set_fault_history()
    sim.close()
