"""qram_run_static: the allocation-free entry point.

Callers that must not allocate device memory while they run (a fixed
device-memory plan, another framework's allocator they may not go around)
pass every input and output as device memory and get the per-CTA scratch
from the library's fixed static device array.  This test calls it through
the C ABI and checks it against qram_run_pruned / qram_run_full (which
allocate their scratch) on two calls in a row: the static array keeps the
previous call's contents, so the second call also checks that the entry
point resets what must start at zero.  It sits in its own file, collected
last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _lib():
    from paper_2609_34935_b300 import load_library
    L = load_library()
    vp, i32, u32, u64, f64 = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
    L.qram_run_static.argtypes = [C.c_int, i32, i32, i32, i32, vp, vp, vp, vp, vp, u64, u64, u32, vp, f64, vp, vp]
    L.qram_run_static.restype = C.c_int
    return L


def _dev(p):
    mem = torch.tensor(np.asarray(p.memory, np.uint8), device="cuda:0")
    addr = torch.tensor(np.asarray(p.addr, np.uint32).astype(np.int64), device="cuda:0").to(torch.int32)
    bus = torch.tensor(np.asarray(p.bus, np.uint32).astype(np.int64), device="cuda:0").to(torch.int32)
    re = torch.tensor(np.ascontiguousarray(np.asarray(p.amp).real), device="cuda:0")
    im = torch.tensor(np.ascontiguousarray(np.asarray(p.amp).imag), device="cuda:0")
    return mem, addr, bus, re, im


def _static(L, mode, p, seed, traj0, g, gmax):
    mem, addr, bus, re, im = _dev(p)
    out = torch.full((g.numel(), 48), 0xAB, dtype=torch.uint8, device="cuda:0")
    rc = L.qram_run_static(mode, p.encoding, p.n, p.k, len(p.addr), mem.data_ptr(), addr.data_ptr(), bus.data_ptr(),
                           re.data_ptr(), im.data_ptr(), seed, traj0, g.numel(), g.data_ptr(), gmax, out.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, out


def _same(a, b):
    for f in ("status", "bad", "ref", "ncand", "explicit_comps", "jumps", "first_jump_slice", "jump_sites", "q_ground"):
        assert np.array_equal(a[f], b[f]), f
    for f in ("fidelity", "fidelity_unsampled", "p_ground"):
        assert np.max(np.abs(a[f] - b[f])) < TOL, f


@pytest.mark.parametrize("enc,n,k,gamma,mode", [(1, 6, 2, 5e-3, 0), (0, 8, 1, 2e-3, 0), (1, 5, 3, 3e-2, 1)])
def test_static_entry_point_matches_allocating_one(enc, n, k, gamma, mode):
    import workloads as W
    from paper_2609_34935_b300 import QramSim
    L = _lib()
    p = W.data_loading(enc, n, k, seed=77 + n)
    seed, traj0, nt = 9001, 123, 700
    g = torch.full((nt,), gamma, dtype=torch.float64, device="cuda:0")
    sim = QramSim(p, seed=seed, device=0)
    ref = QramSim.results(sim.run("pruned" if mode == 0 else "full", traj0, g))
    sim.close()
    assert np.all(ref["status"] == 0)
    for _ in range(2):                      # two calls in a row share the static array
        rc, out = _static(L, mode, p, seed, traj0, g, 0.05)
        assert rc == 0
        _same(QramSim.results(out), ref)


def test_static_entry_point_rejects_oversize():
    import workloads as W
    L = _lib()
    big = W.data_loading(1, 14, 8, seed=1)                    # 16384 x 256 components: beyond 32 MiB
    g = torch.full((4,), 1e-3, dtype=torch.float64, device="cuda:0")
    rc, _ = _static(L, 0, big, 1, 0, g, 1e-2)
    assert rc == 8                                            # QRAM_E_TOOBIG
    p = W.data_loading(1, 6, 2, seed=1)
    rc, _ = _static(L, 0, p, 1, 0, g, 0.9)                    # gamma_max beyond the damping-rate limit
    assert rc == 1                                            # QRAM_E_ARG


def _corrupt(p, kind):
    p.addr, p.bus, p.memory, p.amp = p.addr.copy(), p.bus.copy(), p.memory.copy(), p.amp.copy()
    if kind == "duplicate_address":
        p.addr[3] = p.addr[2]
    elif kind == "address_range":
        p.addr[3] = 1 << p.n
    elif kind == "bus_range":
        p.bus[2] = 1 << p.k
    elif kind == "memory_range":
        p.memory[5] = 1 << p.k
    elif kind == "norm":
        p.amp *= 1.01
    elif kind == "nan_amplitude":
        p.amp[0] = complex(float("nan"), 0.0)
    return p


@pytest.mark.parametrize("kind", ["duplicate_address", "address_range", "bus_range", "memory_range", "norm",
                                  "nan_amplitude"])
def test_static_entry_point_rejects_bad_input(kind):
    """Inputs live in device memory, so they are checked on the device before
    the trajectory kernel reads them: every trajectory reports QRAM_E_ARG."""
    import workloads as W
    from paper_2609_34935_b300 import QramSim
    L = _lib()
    bad = _corrupt(W.data_loading(1, 4, 2, seed=2), kind)
    g = torch.full((4,), 1e-2, dtype=torch.float64, device="cuda:0")
    rc, out = _static(L, 0, bad, 1, 0, g, 1e-2)
    assert rc == 0
    assert np.all(QramSim.results(out)["status"] == 1)        # QRAM_E_ARG on every trajectory


def test_static_entry_point_reports_capacity_without_writing_past_out():
    """A damping rate far above gamma_max overflows the candidate scratch
    sized for gamma_max: the trajectory reports QRAM_E_CAP, the others are
    unaffected, and nothing is written past the caller's output rows."""
    import workloads as W
    from paper_2609_34935_b300 import QramSim
    L = _lib()
    p = W.data_loading(1, 8, 2, seed=5)
    mem, addr, bus, re, im = _dev(p)
    nt, guard = 6, 4
    g = torch.full((nt,), 1e-4, dtype=torch.float64, device="cuda:0")
    g[2] = 0.3
    buf = torch.full((nt + guard, 48), 0xAB, dtype=torch.uint8, device="cuda:0")
    rc = L.qram_run_static(0, p.encoding, p.n, p.k, len(p.addr), mem.data_ptr(), addr.data_ptr(), bus.data_ptr(),
                           re.data_ptr(), im.data_ptr(), 11, 0, nt, g.data_ptr(), 1e-4, buf.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0
    res = QramSim.results(buf[:nt])
    assert res["status"][2] == 6                              # QRAM_E_CAP
    assert np.all(np.delete(res["status"], 2) == 0)
    assert bool(torch.all(buf[nt:] == 0xAB))
