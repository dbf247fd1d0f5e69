"""ctypes wrapper of the C oracle (``qram_oracle.c``).  Test infrastructure only.

The shared library is compiled with gcc into ``oracle/liboracle.so`` by
``build()`` (also called from ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qram_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

OK, E_ARG, E_OOM, E_SCHED, E_CAP = 0, 1, 2, 3, 4
DAMPING, DEPHASING, HEATING = 0, 1, 2   # the per-slice channel (amplitude damping; phase damping; heating)
G_LOAD, G_UNLOAD, G_BUS, G_ISWAP, G_CSWAP, G_FETCH = 1, 2, 3, 4, 5, 6
GATE_NAMES = {1: "load", 2: "unload", 3: "bus", 4: "iswap", 5: "cswap", 6: "fetch"}


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


class _Problem(C.Structure):
    _fields_ = [("encoding", C.c_int32), ("n", C.c_int32), ("k", C.c_int32),
                ("memory", C.c_void_p), ("D", C.c_int32),
                ("addr", C.c_void_p), ("bus", C.c_void_p),
                ("amp_re", C.c_void_p), ("amp_im", C.c_void_p)]


class _Hist(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("cand_slice", C.c_void_p), ("cand_site", C.c_void_p),
                ("aux_u", C.c_void_p), ("final_u", C.c_double),
                ("nflip", C.c_int32), ("flip_slice", C.c_void_p), ("flip_site", C.c_void_p),
                ("eps", C.c_double), ("stop_slice", C.c_int32), ("channel", C.c_int32)]


TRAJ_DTYPE = np.dtype([("fidelity", "f8"), ("fidelity_unsampled", "f8"), ("p_ground", "f8"),
                       ("ncand", "u4"), ("bad", "u4"), ("ref", "i4"),
                       ("jumps", "u4"), ("first_jump_slice", "u4"), ("jump_sites", "u4"),
                       ("q_ground", "u4"), ("status", "u4")])

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, i32, u64, f64 = C.c_void_p, C.c_int32, C.c_uint64, C.c_double
        L.oracle_run.argtypes = [vp, u64, u64, i32, vp, i32, vp]
        L.oracle_run_eps.argtypes = [vp, u64, u64, i32, vp, f64, i32, vp]
        L.oracle_run_ch.argtypes = [vp, u64, u64, i32, vp, f64, i32, i32, vp]
        L.oracle_sample_paulis.argtypes = [vp, u64, u64, f64, vp, vp, vp, i32, vp]
        L.oracle_run_one.argtypes = [vp, u64, u64, f64, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_sample_faults.argtypes = [vp, u64, u64, f64, vp, vp, i32, vp, vp, vp, vp]
        L.oracle_schedule.argtypes = [i32, i32, vp, vp, vp, i32, vp]
        L.oracle_occupancy.argtypes = [vp, vp]
        L.oracle_joint_layer.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, f64, f64, vp, vp, vp, i32, vp]
        L.oracle_bad_range.argtypes = [i32, i32, C.c_uint32, vp, vp]
        L.oracle_bad_range.restype = None
        L.oracle_philox.argtypes = [vp, u64, vp]
        L.oracle_philox.restype = None
        L.oracle_threshold.argtypes = [f64]
        L.oracle_threshold.restype = u64
        L.oracle_gap.argtypes = [u64, f64]
        L.oracle_gap.restype = C.c_uint32
        L.oracle_maxe.restype = i32
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Bound:
    """Keeps the numpy arrays alive while the C struct points into them."""

    def __init__(self, prob):
        self.memory = np.ascontiguousarray(prob.memory, dtype=np.uint8)
        self.addr = np.ascontiguousarray(prob.addr, dtype=np.uint32)
        self.bus = np.ascontiguousarray(prob.bus, dtype=np.uint32)
        amp = np.asarray(prob.amp, dtype=np.complex128)
        self.re = np.ascontiguousarray(amp.real)
        self.im = np.ascontiguousarray(amp.imag)
        self.s = _Problem(prob.encoding, prob.n, prob.k, _ptr(self.memory).value, len(self.addr),
                          _ptr(self.addr).value, _ptr(self.bus).value, _ptr(self.re).value,
                          _ptr(self.im).value)

    @property
    def ref(self):
        return C.byref(self.s)


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != OK:
        raise OracleError(f"{what}: oracle error {rc}")


def run(prob, seed: int, traj0: int, gammas, nthreads: int | None = None, eps: float = 0.0,
        channel: int = DAMPING) -> np.ndarray:
    """Full evolution of trajectories traj0 .. traj0+len(gammas)-1; eps is the
    depolarizing strength per (slice, site), eps < 0 meaning eps = gamma;
    channel: DAMPING (amplitude damping) or DEPHASING (phase damping)."""
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    out = np.zeros(len(g), dtype=TRAJ_DTYPE)
    b = _Bound(prob)
    nt = nthreads or os.cpu_count() or 1
    _check(lib().oracle_run_ch(b.ref, seed, traj0, len(g), _ptr(g), float(eps), int(channel), nt, _ptr(out)),
           "oracle_run")
    return out


@dataclass
class History:
    """A fixed noise history for one trajectory (candidates, optional draws)."""

    cand_slice: list
    cand_site: list
    aux_u: dict | None = None      # slice -> u
    final_u: float | None = None
    flips: list | None = None      # [(slice, site)] X flips (qubit)
    stop_slice: int = 0            # > 0: return the state after this slice's damping layer


@dataclass
class Dump:
    addr: np.ndarray
    bus: np.ndarray
    configs: list          # tuple of (site, level) per component
    amp: np.ndarray        # normalised


def run_one(prob, seed: int, traj: int, gamma: float, hist: History | None = None, cap: int = 1 << 20,
            eps: float = 0.0, channel: int = DAMPING):
    b = _Bound(prob)
    T = 6 * prob.n + 2 * prob.k
    keep = []
    hp = None
    if hist is None and (eps != 0.0 or channel != DAMPING):   # sampled history, options set
        h = _Hist(0, None, None, None, math.nan, 0, None, None, float(eps))
        h.channel = int(channel)
        keep.append(h)
        hp = C.byref(h)
    if hist is not None:
        cs = np.ascontiguousarray(hist.cand_slice, dtype=np.int32)
        cq = np.ascontiguousarray(hist.cand_site, dtype=np.int32)
        au = np.full(T + 1, np.nan)
        for s, u in (hist.aux_u or {}).items():
            au[s] = u
        fl = hist.flips or []
        fs = np.ascontiguousarray([f[0] for f in fl] or [0], dtype=np.int32)
        fq = np.ascontiguousarray([f[1] for f in fl] or [0], dtype=np.int32)
        keep += [cs, cq, au, fs, fq]
        h = _Hist(len(cs), _ptr(cs).value if len(cs) else _ptr(np.zeros(1, np.int32)).value,
                  _ptr(cq).value if len(cq) else None, _ptr(au).value,
                  math.nan if hist.final_u is None else hist.final_u,
                  len(fl), _ptr(fs).value if fl else None, _ptr(fq).value if fl else None)
        h.stop_slice = int(hist.stop_slice)
        h.eps = float(eps)
        h.channel = int(channel)
        if len(cs) == 0:
            z = np.zeros(1, np.int32)
            keep.append(z)
            h.cand_slice = _ptr(z).value
            h.cand_site = _ptr(z).value
        keep.append(h)
        hp = C.byref(h)
    L = lib()
    maxe = L.oracle_maxe()
    while True:
        out = np.zeros(1, dtype=TRAJ_DTYPE)
        ncomp = C.c_int32(0)
        da = np.zeros(cap, np.uint32)
        db = np.zeros(cap, np.uint32)
        dn = np.zeros(cap, np.int32)
        ds = np.zeros(cap * maxe, np.uint32)
        dl = np.zeros(cap * maxe, np.uint8)
        dr = np.zeros(cap, np.float64)
        di = np.zeros(cap, np.float64)
        rc = L.oracle_run_one(b.ref, seed, traj, gamma, hp, _ptr(out), cap, C.byref(ncomp),
                              _ptr(da), _ptr(db), _ptr(dn), _ptr(ds), _ptr(dl), _ptr(dr), _ptr(di))
        if rc == E_CAP:
            cap = int(ncomp.value) + 16
            continue
        _check(rc, "oracle_run_one")
        m = int(ncomp.value)
        configs = []
        for r in range(m):
            ne = int(dn[r])
            configs.append(tuple((int(ds[r * maxe + e]), int(dl[r * maxe + e])) for e in range(ne)))
        return out[0], Dump(da[:m].copy(), db[:m].copy(), configs, dr[:m] + 1j * di[:m])


def sample_paulis(prob, seed: int, traj: int, eps: float):
    """Depolarizing fault events (slice, site, operator index) of one trajectory."""
    b = _Bound(prob)
    cap = 1 << 16
    while True:
        sl = np.zeros(cap, np.int32)
        st = np.zeros(cap, np.int32)
        ty = np.zeros(cap, np.int32)
        ne = C.c_int32(0)
        rc = lib().oracle_sample_paulis(b.ref, seed, traj, float(eps), _ptr(sl), _ptr(st), _ptr(ty), cap, C.byref(ne))
        if rc == E_CAP:
            cap = int(ne.value) + 16
            continue
        _check(rc, "oracle_sample_paulis")
        m = int(ne.value)
        return sl[:m].copy(), st[:m].copy(), ty[:m].copy()


def sample_faults(prob, seed: int, traj: int, gamma: float):
    """Candidate list (slice, site), bad bitmap over addresses, B and reference index."""
    b = _Bound(prob)
    cap = 1 << 16
    while True:
        sl = np.zeros(cap, np.int32)
        st = np.zeros(cap, np.int32)
        nc = C.c_int32(0)
        bad = np.zeros(1 << prob.n, np.uint8)
        B = C.c_uint32(0)
        ref = C.c_int32(0)
        rc = lib().oracle_sample_faults(b.ref, seed, traj, gamma, _ptr(sl), _ptr(st), cap,
                                        C.byref(nc), _ptr(bad), C.byref(B), C.byref(ref))
        if rc == E_CAP:
            cap = int(nc.value) + 1
            continue
        _check(rc, "oracle_sample_faults")
        m = int(nc.value)
        return sl[:m].copy(), st[:m].copy(), bad, int(B.value), int(ref.value)


def schedule(n: int, k: int):
    cap = 8192
    kind = np.zeros(cap, np.int32)
    par = np.zeros(cap, np.int32)
    sl = np.zeros(cap, np.int32)
    cnt = C.c_int(0)
    _check(lib().oracle_schedule(n, k, _ptr(kind), _ptr(par), _ptr(sl), cap, C.byref(cnt)), "schedule")
    m = cnt.value
    return [(int(sl[i]), GATE_NAMES[int(kind[i])], int(par[i])) for i in range(m)]


def schedule_rc(n: int, k: int) -> int:
    cap = 8192
    kind = np.zeros(cap, np.int32)
    cnt = C.c_int(0)
    return lib().oracle_schedule(n, k, _ptr(kind), _ptr(kind), _ptr(kind), cap, C.byref(cnt))


def occupancy(prob) -> np.ndarray:
    T = 6 * prob.n + 2 * prob.k
    M = 2 * ((1 << prob.n) - 1)
    occ = np.zeros(T * M, np.uint8)
    b = _Bound(prob)
    _check(lib().oracle_occupancy(b.ref, _ptr(occ)), "occupancy")
    return occ.reshape(T, M)


def joint_layer(comps, cand, gamma: float, u: float, channel: int = DAMPING, levels=None):
    """One joint layer (amplitude damping, dephasing or heating) on an explicit state;
    levels: heating only, the target level (1 = L / excited, 2 = R) of each candidate in sorted order.

    comps: list of (addr, bus, config, amp) with config a tuple of (site, level).
    Returns (new comps, J as tuple of (site, level))."""
    L = lib()
    maxe = L.oracle_maxe()
    m = len(comps)
    addr = np.array([c[0] for c in comps], np.uint32)
    bus = np.array([c[1] for c in comps], np.uint32)
    ne = np.array([len(c[2]) for c in comps], np.int32)
    sites = np.zeros(m * maxe, np.uint32)
    lvls = np.zeros(m * maxe, np.uint8)
    for r, c in enumerate(comps):
        for e, (q, lv) in enumerate(c[2]):
            sites[r * maxe + e] = q
            lvls[r * maxe + e] = lv
    re = np.array([complex(c[3]).real for c in comps], np.float64)
    im = np.array([complex(c[3]).imag for c in comps], np.float64)
    cnd = np.ascontiguousarray(sorted(cand) or [0], dtype=np.int32)
    hl = np.ascontiguousarray([levels[q] for q in sorted(cand)] if levels is not None and len(cand) else [1],
                              dtype=np.uint8)
    nout = C.c_int32(0)
    jn = C.c_int32(0)
    js = np.zeros(maxe, np.uint32)
    jl = np.zeros(maxe, np.uint8)
    _check(L.oracle_joint_layer(m, _ptr(addr), _ptr(bus), _ptr(ne), _ptr(sites), _ptr(lvls), _ptr(re),
                                _ptr(im), C.byref(nout), _ptr(cnd), len(cand), gamma, u,
                                C.byref(jn), _ptr(js), _ptr(jl), int(channel), _ptr(hl)), "joint_layer")
    out = []
    for r in range(nout.value):
        cfg = tuple((int(sites[r * maxe + e]), int(lvls[r * maxe + e])) for e in range(int(ne[r])))
        out.append((int(addr[r]), int(bus[r]), cfg, complex(re[r], im[r])))
    J = tuple((int(js[j]), int(jl[j])) for j in range(jn.value))
    return out, J


def bad_range(encoding: int, n: int, v: int):
    lo = C.c_uint32(0)
    hi = C.c_uint32(0)
    lib().oracle_bad_range(encoding, n, v, C.byref(lo), C.byref(hi))
    return int(lo.value), int(hi.value)


def philox(ctr, seed: int):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().oracle_philox(_ptr(c), seed, _ptr(o))
    return [int(x) for x in o]


def gap(u: int, gamma: float) -> int:
    """Geometric gap of a 64-bit uniform word: non-candidate sites before the
    next candidate (the fault stream of the random-number convention)."""
    return int(lib().oracle_gap(int(u), float(gamma)))


def threshold(gamma: float) -> int:
    return int(lib().oracle_threshold(gamma))
