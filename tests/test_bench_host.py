"""Host logic of bench.py (no GPU): the DRAM-traffic record is used only
while the kernel sources it was taken on are unchanged, the source hash
covers the kernel sources, and the workload configurations are the ones the
benchmark documents."""
import json
import os

import bench
import workloads as W


def test_traffic_record_needs_matching_sources(tmp_path, monkeypatch):
    """The small-case record's bytes per trajectory scale to the step's
    trajectories, and only while the kernel sources are the recorded ones."""
    rec = tmp_path / "traffic.json"
    h = bench._kernel_sources_hash()
    rec.write_text(json.dumps({"dram_bytes_per_trajectory": 123.0, "sources_sha256": h}))
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    assert bench._traffic_per_step() == 123.0 * bench.NTRAJ
    rec.write_text(json.dumps({"dram_bytes_per_trajectory": 123.0, "sources_sha256": "0" * 64}))
    assert bench._traffic_per_step() is None
    rec.write_text(json.dumps({"dram_bytes_per_step_launch": 123, "sources_sha256": h}))   # full-size record: unused
    assert bench._traffic_per_step() is None
    rec.write_text("not json")
    assert bench._traffic_per_step() is None
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(tmp_path / "missing.json"))
    assert bench._traffic_per_step() is None


def test_source_hash_covers_the_kernel_sources(tmp_path, monkeypatch):
    # a copy of the tree whose kernel source differs by one byte hashes differently
    import shutil
    src = os.path.join(bench.ROOT, "paper_2609_34935_b300", "csrc")
    dst = tmp_path / "paper_2609_34935_b300" / "csrc"
    shutil.copytree(src, dst)
    (tmp_path / "include").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "include", "qram_sim.h"), tmp_path / "include" / "qram_sim.h")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_sources_hash()
    k = dst / "qram_kernels.cu"
    k.write_bytes(k.read_bytes() + b"\n")
    assert bench._kernel_sources_hash() != h0


def test_workload_configurations():
    assert (bench.N, bench.K, bench.NTRAJ, bench.BATCH) == (12, 4, 100_000, 1000)
    assert (bench.G_LO, bench.G_HI) == (1e-5, 1e-2)
    got = [(enc, n, k, tuple(g), nt, tuple(s)) for _, enc, n, k, g, nt, s in bench.CONFIGS]
    assert got == [
        (W.QUTRIT, 3, 1, (1e-3,), 1000, (1001,)),
        (W.QUBIT, 6, 1, (1e-4, 1e-3, 1e-2), 10_000, (2001, 2002, 2003)),
        (W.QUTRIT, 10, 1, (1e-3,), 100_000, (3001,)),
    ]
    # the bench's gammas: one log-uniform value per batch of 1000, inside the range
    g = bench._gammas()
    assert len(g) == bench.NTRAJ
    assert g.min() >= bench.G_LO and g.max() <= bench.G_HI
    assert all(len(set(g[b:b + bench.BATCH])) == 1 for b in range(0, bench.NTRAJ, bench.BATCH))
