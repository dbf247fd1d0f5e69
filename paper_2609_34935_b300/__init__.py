"""B300 (sm_103a) trajectory simulator for amplitude-damped bucket-brigade QRAM
with branch pruning (arXiv 2609.34935).

This module is a thin ctypes binding over the C ABI of ``include/qram_sim.h``
(shared library ``libqram_b300.so``, built by ``build.py``).  It only
marshals arguments: every step of the simulation runs in the CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: if
the library is missing or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["QramSim", "QramServer", "QramBatch", "RESULT_DTYPE", "QramError", "load_library", "QUTRIT", "QUBIT"]

QUTRIT, QUBIT = 0, 1
OK = 0
ERRORS = {1: "E_ARG", 2: "E_OOM", 3: "E_CUDA", 4: "E_TIMEOUT", 5: "E_BUSY", 6: "E_CAP", 7: "E_STATE"}

RESULT_DTYPE = np.dtype([("fidelity", "<f8"), ("fidelity_unsampled", "<f8"), ("p_ground", "<f8"),
                         ("bad", "<u4"), ("ref", "<i4"), ("ncand", "<u4"), ("explicit_comps", "<u4"),
                         ("jumps", "<u2"), ("first_jump_slice", "<u2"), ("jump_sites", "<u2"),
                         ("q_ground", "u1"), ("status", "u1")])
assert RESULT_DTYPE.itemsize == 48


class QramError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {ERRORS.get(code, code)}")
        self.code = code


SAMPLER_VERSION = 2          # candidate sampler of the library (geometric gaps)


class _Problem(C.Structure):
    _fields_ = [("encoding", C.c_int32), ("n", C.c_int32), ("k", C.c_int32), ("memory", C.c_void_p),
                ("num_branches", C.c_int32), ("addr", C.c_void_p), ("bus", C.c_void_p),
                ("amp_re", C.c_void_p), ("amp_im", C.c_void_p), ("seed", C.c_uint64),
                ("sampler_version", C.c_uint32)]


class _Request(C.Structure):
    _fields_ = [("problem", _Problem), ("traj0", C.c_uint64), ("ntraj", C.c_uint32),
                ("gamma", C.c_void_p), ("mode", C.c_int32)]


class _Completion(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int32), ("ntraj", C.c_uint32),
                ("mean_fidelity", C.c_double), ("stderr_fidelity", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_finish", C.c_double),
                ("device_bytes", C.c_uint64)]


_lib = None


def load_library(build_if_missing: bool = True):
    """Load libqram_b300.so (building it with nvcc when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        try:
            path = _build.build()
        except Exception as e:  # pragma: no cover
            if not os.path.exists(path):
                raise RuntimeError(f"cannot build {path}: {e}") from e
    if not os.path.exists(path):
        raise RuntimeError(f"{path} missing: run `python -m paper_2609_34935_b300.build`")
    L = C.CDLL(path)
    vp, u32, u64, i32, f64 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_double
    L.qram_sim_create.argtypes = [vp, C.c_int, vp, C.POINTER(vp)]
    L.qram_sim_destroy.argtypes = [vp]
    L.qram_sim_destroy.restype = None
    L.qram_sample_faults.argtypes = [vp, u64, u32, vp, u32, vp, vp, vp, vp, vp]
    L.qram_run_pruned.argtypes = [vp, u64, u32, vp, vp]
    L.qram_run_full.argtypes = [vp, u64, u32, vp, vp]
    L.qram_set_fault_history.argtypes = [vp, u32, vp, vp]
    L.qram_fidelity.argtypes = [vp, vp, u32, C.POINTER(f64), C.POINTER(f64)]
    L.qram_dump_state.argtypes = [vp, C.c_int, u64, f64, u32, vp, vp, vp, vp, vp, C.POINTER(u32)]
    L.qram_set_gamma_bound.argtypes = [vp, f64]
    L.qram_set_launch_ctas.argtypes = [vp, u32]
    L.qram_sync.argtypes = [vp]
    L.qram_launch_count.argtypes = [vp]
    L.qram_launch_count.restype = u64
    L.qram_work_counters.argtypes = [vp, vp, C.c_int]
    L.qram_set_dump_weight.argtypes = [vp, C.c_int]
    L.qram_set_depolarizing.argtypes = [vp, C.c_double, C.c_int]
    L.qram_set_channel.argtypes = [vp, C.c_int]
    L.qram_server_create.argtypes = [C.c_size_t, C.c_int, u32, C.POINTER(vp)]
    L.qram_server_submit.argtypes = [vp, vp, C.POINTER(u64)]
    L.qram_server_estimate.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.qram_server_poll.argtypes = [vp, vp, u32, C.POINTER(u32)]
    L.qram_server_results.argtypes = [vp, u64, vp, u32]
    L.qram_server_cancel.argtypes = [vp, u64]
    L.qram_server_drain.argtypes = [vp, f64]
    L.qram_server_destroy.argtypes = [vp]
    L.qram_server_destroy.restype = None
    L.qram_graph_create.argtypes = [vp, C.c_int, u32, vp, vp, vp, C.POINTER(vp)]
    L.qram_graph_launch.argtypes = [vp]
    L.qram_graph_destroy.argtypes = [vp]
    L.qram_graph_destroy.restype = None
    L.qram_batch_create.argtypes = [vp, u32, C.c_int, C.c_int, vp, vp, vp, vp, C.POINTER(vp)]
    L.qram_batch_launch.argtypes = [vp]
    L.qram_batch_grid.argtypes = [vp]
    L.qram_batch_destroy.argtypes = [vp]
    L.qram_batch_destroy.restype = None
    L.qram_set_variant.argtypes = [vp, C.c_int]
    L.qram_get_variant.argtypes = [vp]
    L.qram_autotune.argtypes = [vp, C.c_int, f64, u32, u64, C.POINTER(C.c_int), C.POINTER(C.c_float)]
    L.qram_measure_peaks.argtypes = [C.c_int, C.POINTER(f64), C.POINTER(f64)]
    L.qram_strerror.argtypes = [C.c_int]
    L.qram_strerror.restype = C.c_char_p
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != OK:
        raise QramError(rc, what)


def _dptr(t) -> int:
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
    return t.data_ptr()


class QramSim:
    """One QRAM problem resident on a CUDA device.

    ``problem`` needs ``encoding, n, k, memory, addr, bus, amp`` (numpy);
    ``seed`` keys the Philox streams."""

    def __init__(self, problem, seed: int, device: int = 0, stream=None):
        import torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("QramSim needs a CUDA device (no CPU fallback)")
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.problem = problem
        self.n, self.k, self.encoding = int(problem.n), int(problem.k), int(problem.encoding)
        mem = np.ascontiguousarray(problem.memory, dtype=np.uint8)
        addr = np.ascontiguousarray(problem.addr, dtype=np.uint32)
        bus = np.ascontiguousarray(problem.bus, dtype=np.uint32)
        amp = np.asarray(problem.amp, dtype=np.complex128)
        re = np.ascontiguousarray(amp.real)
        im = np.ascontiguousarray(amp.imag)
        p = _Problem(self.encoding, self.n, self.k, mem.ctypes.data, len(addr), addr.ctypes.data,
                     bus.ctypes.data, re.ctypes.data, im.ctypes.data, int(seed) & (2 ** 64 - 1), SAMPLER_VERSION)
        h = C.c_void_p()
        _check(self.lib.qram_sim_create(C.byref(p), device, self.stream.cuda_stream, C.byref(h)), "qram_sim_create")
        self.h = h
        self._hist = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.qram_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def D(self) -> int:
        return int(len(self.problem.addr))

    def _gam(self, gammas):
        import torch
        g = torch.as_tensor(gammas, dtype=torch.float64)
        if not g.is_cuda:
            g = g.to(f"cuda:{self.device}")
        return g.contiguous()

    def run(self, mode: str, traj0: int, gammas, out=None):
        """Launch trajectories traj0..traj0+len(gammas)-1; returns a uint8
        device tensor [ntraj, 48] (layout RESULT_DTYPE)."""
        import torch
        g = self._gam(gammas)
        nt = g.numel()
        if out is None:
            out = torch.empty((nt, RESULT_DTYPE.itemsize), dtype=torch.uint8, device=g.device)
        fn = self.lib.qram_run_pruned if mode == "pruned" else self.lib.qram_run_full
        _check(fn(self.h, traj0, nt, _dptr(g), _dptr(out)), f"qram_run_{mode}")
        return out

    def run_pruned(self, traj0: int, gammas, out=None):
        return self.run("pruned", traj0, gammas, out)

    def run_full(self, traj0: int, gammas, out=None):
        return self.run("full", traj0, gammas, out)

    @staticmethod
    def results(raw) -> np.ndarray:
        """Copy a result tensor to the host as a structured numpy array."""
        return raw.cpu().numpy().view(RESULT_DTYPE).reshape(-1)

    def sample_faults(self, traj0: int, gammas, cap: int = 1 << 14):
        import torch
        g = self._gam(gammas)
        nt = g.numel()
        W = ((1 << self.n) + 31) // 32
        dev = g.device
        cand = torch.zeros((nt, cap), dtype=torch.int32, device=dev)
        ncand = torch.zeros(nt, dtype=torch.int32, device=dev)
        bits = torch.zeros((nt, W), dtype=torch.int32, device=dev)
        bad = torch.zeros(nt, dtype=torch.int32, device=dev)
        ref = torch.zeros(nt, dtype=torch.int32, device=dev)
        _check(self.lib.qram_sample_faults(self.h, traj0, nt, _dptr(g), cap, _dptr(cand), _dptr(ncand),
                                           _dptr(bits), _dptr(bad), _dptr(ref)), "qram_sample_faults")
        return dict(cand=cand, ncand=ncand, bad_bits=bits, bad=bad, ref=ref)

    def set_fault_history(self, cand=None, off=None):
        """cand: int32 device tensor of packed (slice << 16 | site); off: int32 [nhist+1]."""
        if cand is None:
            _check(self.lib.qram_set_fault_history(self.h, 0, None, None), "qram_set_fault_history")
            self._hist = None
            return
        self._hist = (cand, off)          # keep alive while set
        _check(self.lib.qram_set_fault_history(self.h, off.numel() - 1, _dptr(cand), _dptr(off)),
               "qram_set_fault_history")

    def fidelity(self, raw):
        m, s = C.c_double(), C.c_double()
        _check(self.lib.qram_fidelity(self.h, _dptr(raw), raw.shape[0], C.byref(m), C.byref(s)), "qram_fidelity")
        return m.value, s.value

    def dump_state(self, mode: str, traj: int, gamma: float, cap: int = 1 << 18, w_max: int = -1):
        """Final normalised state of one trajectory; w_max >= 0 keeps only the
        good-branch output words within that Hamming distance of the ideal
        word (low-weight truncation)."""
        _check(self.lib.qram_set_dump_weight(self.h, int(w_max)), "qram_set_dump_weight")
        while True:
            addr = np.zeros(cap, np.uint32)
            bus = np.zeros(cap, np.uint32)
            hsh = np.zeros(cap, np.uint64)
            re = np.zeros(cap, np.float64)
            im = np.zeros(cap, np.float64)
            cnt = C.c_uint32(0)
            rc = self.lib.qram_dump_state(self.h, 0 if mode == "pruned" else 1, traj, gamma, cap,
                                          addr.ctypes.data, bus.ctypes.data, hsh.ctypes.data, re.ctypes.data,
                                          im.ctypes.data, C.byref(cnt))
            if rc == 6 and cnt.value > cap:
                cap = cnt.value + 16
                continue
            _check(rc, "qram_dump_state")
            m = cnt.value
            return addr[:m], bus[:m], hsh[:m], re[:m] + 1j * im[:m]

    def set_depolarizing(self, eps: float, eps_equals_gamma: bool = False):
        """Depolarizing faults of strength eps per (slice, site) on top of the
        damping (eps_equals_gamma: each trajectory's damping rate)."""
        _check(self.lib.qram_set_depolarizing(self.h, float(eps), 1 if eps_equals_gamma else 0),
               "qram_set_depolarizing")

    def set_channel(self, channel: str):
        """The per-slice channel: "damping" (amplitude damping, the default),
        "dephasing" (phase damping with the same no-jump operator) or
        "heating" (diagonal no-jump operator on the ground level, jumps to the
        excited levels; every branch explicit)."""
        _check(self.lib.qram_set_channel(self.h, {"damping": 0, "dephasing": 1, "heating": 2}[channel]),
               "qram_set_channel")

    def set_gamma_bound(self, gmax: float):
        _check(self.lib.qram_set_gamma_bound(self.h, gmax), "qram_set_gamma_bound")

    def set_launch_ctas(self, nctas: int):
        _check(self.lib.qram_set_launch_ctas(self.h, nctas), "qram_set_launch_ctas")

    def graph(self, mode: str, gammas, out, traj0_dev):
        """Capture one batched launch into a CUDA graph (see qram_graph_create);
        returns a callable that replays it on the simulator's stream."""
        h = C.c_void_p()
        _check(self.lib.qram_graph_create(self.h, 0 if mode == "pruned" else 1, gammas.numel(), _dptr(gammas),
                                          _dptr(out), _dptr(traj0_dev), C.byref(h)), "qram_graph_create")
        lib = self.lib

        class _Graph:
            def __init__(self, handle, keep):
                self.h, self.keep = handle, keep

            def __call__(self):
                _check(lib.qram_graph_launch(self.h), "qram_graph_launch")

            def close(self):
                if self.h:
                    lib.qram_graph_destroy(self.h)
                    self.h = None

            def __del__(self):
                try:
                    self.close()
                except Exception:
                    pass
        return _Graph(h, (gammas, out, traj0_dev))

    def set_variant(self, threads: int):
        _check(self.lib.qram_set_variant(self.h, threads), "qram_set_variant")

    @property
    def variant(self) -> int:
        return int(self.lib.qram_get_variant(self.h))

    def autotune(self, mode: str = "pruned", gamma: float = 3e-3, ntraj: int = 2000, cache: str | None = None):
        """Pick the fastest launch variant for this problem (threads per CTA).
        With `cache` (a JSON path) the choice is looked up / stored under the
        key (encoding, n, k, decade of gamma)."""
        import json
        import math
        key = f"{self.encoding}:{self.n}:{self.k}:{mode}:1e{int(math.floor(math.log10(max(gamma, 1e-12))))}"
        table = {}
        if cache and os.path.exists(cache):
            try:
                table = json.load(open(cache))
            except Exception:
                table = {}
        if key in table:
            self.set_variant(int(table[key]["threads"]))
            return int(table[key]["threads"])
        best = C.c_int()
        ms = C.c_float()
        _check(self.lib.qram_autotune(self.h, 0 if mode == "pruned" else 1, gamma, ntraj, 1 << 40, C.byref(best),
                                      C.byref(ms)), "qram_autotune")
        if cache:
            table[key] = {"threads": int(best.value), "ms": float(ms.value), "ntraj": ntraj}
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return int(best.value)

    def sync(self):
        _check(self.lib.qram_sync(self.h), "qram_sync")

    @property
    def launch_count(self) -> int:
        return int(self.lib.qram_launch_count(self.h))

    def work_counters(self, reset: bool = False) -> dict:
        """Work of the trajectory launches since creation or the last reset:
        fault-stream draws, explicit component-slices, closed-form
        branch-epochs, explicit component-epochs, and the component-slices
        (epochs) taken by the two-path, register generic, memory generic
        (off-path) forms (waits for the stream)."""
        o = np.zeros(8, np.uint64)
        _check(self.lib.qram_work_counters(self.h, o.ctypes.data, 1 if reset else 0), "qram_work_counters")
        names = ("draws", "comp_slices", "branch_epochs", "comp_epochs", "two_path_slices", "reg_generic_slices",
                 "mem_generic_slices", "offpath_comp_epochs")
        return {nm: int(v) for nm, v in zip(names, o)}


class QramBatch:
    """One persistent launch over several problems (qram_batch_create): a
    CUDA graph replayed by calling the object.  ``sims``: QramSim objects on
    one device, each with a damping-rate bound; ``gammas``/``outs``: device
    tensors per problem (float64 rates; uint8 [ntraj, 48] results);
    ``traj0s``: first trajectory index per problem."""

    def __init__(self, sims, mode: str, traj0s, gammas, outs, threads: int = 0):
        self.lib = load_library()
        n = len(sims)
        hs = (C.c_void_p * n)(*[s.h for s in sims])
        t0 = (C.c_uint64 * n)(*[int(t) for t in traj0s])
        nt = (C.c_uint32 * n)(*[int(g.numel()) for g in gammas])
        gp = (C.c_void_p * n)(*[_dptr(g) for g in gammas])
        op = (C.c_void_p * n)(*[_dptr(o) for o in outs])
        for g, o in zip(gammas, outs):
            assert o.shape[0] == g.numel() and o.shape[1] == RESULT_DTYPE.itemsize
        h = C.c_void_p()
        _check(self.lib.qram_batch_create(hs, n, 0 if mode == "pruned" else 1, int(threads), t0, nt, gp, op,
                                          C.byref(h)), "qram_batch_create")
        self.h = h
        self._keep = (list(sims), list(gammas), list(outs))

    @property
    def grid(self) -> int:
        return int(self.lib.qram_batch_grid(self.h))

    def __call__(self):
        _check(self.lib.qram_batch_launch(self.h), "qram_batch_launch")

    def close(self):
        if getattr(self, "h", None):
            self.lib.qram_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_peaks(device: int = 0) -> dict:
    """Measured FP64 FMA (FLOP/s) and 32-bit integer add/logic (ops/s)
    throughput of the device (qram_measure_peaks): roofline denominators."""
    L = load_library()
    fp, it = C.c_double(), C.c_double()
    _check(L.qram_measure_peaks(device, C.byref(fp), C.byref(it)), "qram_measure_peaks")
    return {"fp64_flops": fp.value, "int32_ops": it.value}


class QramServer:
    """Continuous-batching serving loop (native scheduler thread in the library)."""

    def __init__(self, mem_budget: int, device: int = 0, max_active: int = 4):
        self.lib = load_library()
        h = C.c_void_p()
        _check(self.lib.qram_server_create(mem_budget, device, max_active, C.byref(h)), "qram_server_create")
        self.h = h

    @staticmethod
    def _request(problem, seed, traj0, gammas, mode):
        keep = []
        mem = np.ascontiguousarray(problem.memory, dtype=np.uint8)
        addr = np.ascontiguousarray(problem.addr, dtype=np.uint32)
        bus = np.ascontiguousarray(problem.bus, dtype=np.uint32)
        amp = np.asarray(problem.amp, dtype=np.complex128)
        re = np.ascontiguousarray(amp.real)
        im = np.ascontiguousarray(amp.imag)
        g = np.ascontiguousarray(gammas, dtype=np.float64)
        keep += [mem, addr, bus, re, im, g]
        p = _Problem(int(problem.encoding), int(problem.n), int(problem.k), mem.ctypes.data, len(addr),
                     addr.ctypes.data, bus.ctypes.data, re.ctypes.data, im.ctypes.data,
                     int(seed) & (2 ** 64 - 1), SAMPLER_VERSION)
        return _Request(p, int(traj0), len(g), g.ctypes.data, int(mode)), keep

    def submit(self, problem, seed: int, traj0: int, gammas, mode: int = 0) -> int:
        req, keep = self._request(problem, seed, traj0, gammas, mode)
        rid = C.c_uint64()
        _check(self.lib.qram_server_submit(self.h, C.byref(req), C.byref(rid)), "qram_server_submit")
        del keep
        return int(rid.value)

    def estimate(self, problem, ntraj: int, gamma: float = 1e-2) -> int:
        req, keep = self._request(problem, 0, 0, np.full(ntraj, gamma), 0)
        b = C.c_size_t()
        _check(self.lib.qram_server_estimate(self.h, C.byref(req), C.byref(b)), "qram_server_estimate")
        return int(b.value)

    def poll(self, max_items: int = 4096):
        buf = (_Completion * max_items)()
        cnt = C.c_uint32()
        _check(self.lib.qram_server_poll(self.h, buf, max_items, C.byref(cnt)), "qram_server_poll")
        return [{f: getattr(buf[i], f) for f, _ in _Completion._fields_} for i in range(cnt.value)]

    def results(self, rid: int, ntraj: int):
        out = np.zeros(ntraj, dtype=RESULT_DTYPE)
        _check(self.lib.qram_server_results(self.h, rid, out.ctypes.data, ntraj), "qram_server_results")
        return out

    def cancel(self, rid: int):
        _check(self.lib.qram_server_cancel(self.h, rid), "qram_server_cancel")

    def drain(self, timeout_s: float) -> bool:
        rc = self.lib.qram_server_drain(self.h, timeout_s)
        if rc == 4:
            return False
        _check(rc, "qram_server_drain")
        return True

    def close(self):
        if getattr(self, "h", None):
            self.lib.qram_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
