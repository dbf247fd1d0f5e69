"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/qram_sim.h declares; the product path refuses to run
without CUDA (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(qram_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2609_34935_b300 import load_library
    lib = load_library()
    names = _declared()
    assert {"qram_sim_create", "qram_run_pruned", "qram_run_full", "qram_sample_faults", "qram_fidelity"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert lib.qram_strerror(6) == b"per-trajectory capacity exceeded"


def test_create_rejects_bad_problems_without_gpu():
    import numpy as np
    import workloads as W
    import paper_2609_34935_b300 as Q
    lib = Q.load_library()
    p = W.data_loading(W.QUBIT, 3, 4, seed=1)          # k > n
    mem = np.ascontiguousarray(p.memory)
    a = np.ascontiguousarray(p.addr)
    b = np.ascontiguousarray(p.bus)
    re_ = np.ascontiguousarray(p.amp.real)
    im_ = np.ascontiguousarray(p.amp.imag)
    pr = Q._Problem(1, 3, 4, mem.ctypes.data, len(a), a.ctypes.data, b.ctypes.data, re_.ctypes.data,
                    im_.ctypes.data, 1, Q.SAMPLER_VERSION)
    h = ctypes.c_void_p()
    assert lib.qram_sim_create(ctypes.byref(pr), 0, None, ctypes.byref(h)) == 1
    pr.k = 2
    pr.sampler_version = 1                  # the per-node draw is not implemented
    assert lib.qram_sim_create(ctypes.byref(pr), 0, None, ctypes.byref(h)) == 1


def test_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import workloads as W
    from paper_2609_34935_b300 import QramSim
    with pytest.raises(RuntimeError):
        QramSim(W.data_loading(W.QUBIT, 3, 1, seed=1), seed=1)
