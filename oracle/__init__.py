"""CPU oracle for BGPC / D2GC (Tas, Kaya, Saule, arXiv 1701.02628).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's ``cpu_baseline`` / ``--impl reference`` leg may import this
package.  It shares no code with the CUDA path (``paper_1701_02628_gb300``)
and neither imports the other.

The arithmetic lives in plain C (``bgpc_oracle.c``); this module only
marshals numpy arrays.  Graph arguments are any object with the attributes
``n_a, n_b, a_ptr, a_idx, b_ptr, b_idx`` (int32 numpy arrays) and, for the
undirected helpers, ``n, ptr, idx``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from types import SimpleNamespace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "bgpc_oracle.c"), os.path.join(_HERE, "bgpc_oracle.h")]
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

FF, B1, B2, B2X = 0, 1, 2, 3
OK, EINVAL, ENOMEM, EROUNDS, EFIXED, STOPPED = 0, -1, -2, -4, -7, 1
NO_BIG = (1 << 31) - 1  # big_net threshold that disables the reverse first fit


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (no-op when up to date)."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c11",
                           "-Wall", "-o", tmp, _SRC[0]])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER(ctypes.c_int32)
    P64 = ctypes.POINTER(ctypes.c_int64)
    P8 = ctypes.POINTER(ctypes.c_uint8)
    G = [i32, i32, P, P, P, P]
    sig = {
        "orc_seq_color": (G + [P, i32, P], ctypes.c_int),
        "orc_rs_color": (G + [P, i32, i32, i32, i64, i32, i32, i32, i64, i32, i32, P, P,
                              P64, P64, i32, P, P, P], ctypes.c_int),
        "orc_rs_chunks": (G + [P, P, i32, i32, i32, i64, P, i32, i32, P], ctypes.c_int),
        "orc_rs_losers": (G + [P, P, i32, P, i32, P8], ctypes.c_int),
        "orc_conflicts": (G + [P], i64),
        "orc_max_nbor": (G + [P], i32),
        "orc_bruteforce_min": (G, i32),
        "orc_closed_nbhd": ([i32, P, P, P, P], ctypes.c_int),
        "orc_d2_conflicts": ([i32, P, P, P], i64),
        "orc_color_sets": ([i32, P, P, P64], i32),
        "orc_sl_rank": (G + [P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _p64(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _g(g):
    return [int(g.n_a), int(g.n_b), _p(g.a_ptr), _p(g.a_idx), _p(g.b_ptr), _p(g.b_idx)]


def seq_color(g, policy: int = FF, rank=None) -> np.ndarray:
    """O-1: sequential greedy (Alg. 1 on one thread with Alg. 4's gather)."""
    c = np.empty(g.n_a, np.int32)
    r = None if rank is None else _i32(rank)
    rc = _load().orc_seq_color(*_g(g), _p(r), policy, _p(c))
    if rc != OK:
        raise ValueError(f"orc_seq_color failed: {rc}")
    return c


def rs_color(g, policy: int = FF, chunk: int = 64, waves: int = 16, big_net: int = 64,
             rank=None, max_rounds: int = 1 << 30, stop_after_waves: int = 0,
             nthreads: int = 1, max_report: int = 4096, net_rounds: int = 0,
             center_first: bool = False, stop_before_removal: bool = False):
    """O-2: round-synchronous speculative coloring RS(C, Q, T, policy, rank),
    with the first ``net_rounds`` rounds colored net by net (Alg. 8; Alg. 9
    with ``center_first`` for D2GC's closed neighbourhoods).

    Returns a namespace with colors, status, rounds, w_per_round,
    trav_per_round and, when stopped, W (current work queue), m and wave."""
    n = g.n_a
    c = np.empty(n, np.int32)
    rounds = ctypes.c_int32(0)
    m = ctypes.c_int32(0)
    wave = ctypes.c_int32(-1)
    wpr = np.zeros(max_report, np.int64)
    tpr = np.zeros(max_report, np.int64)
    W = np.empty(max(n, 1), np.int32)
    r = None if rank is None else _i32(rank)
    rc = _load().orc_rs_color(*_g(g), _p(r), policy, chunk, waves, big_net, max_rounds,
                              net_rounds, int(bool(center_first)), stop_after_waves,
                              int(bool(stop_before_removal)), nthreads, _p(c),
                              ctypes.byref(rounds),
                              _p64(wpr), _p64(tpr), max_report, _p(W), ctypes.byref(m),
                              ctypes.byref(wave))
    if rc not in (OK, STOPPED, EROUNDS, EFIXED):
        raise ValueError(f"orc_rs_color failed: {rc}")
    nr = min(rounds.value, max_report)
    return SimpleNamespace(colors=c, status=rc, rounds=rounds.value,
                           w_per_round=wpr[:nr].copy(), trav_per_round=tpr[:nr].copy(),
                           W=W[:m.value].copy(), m=m.value, wave=wave.value)


def rs_chunks(g, S, W, chunks, policy: int = FF, chunk: int = 64, big_net: int = 64,
              nthreads: int = 1):
    """One wave step of O-2: colors of the listed chunks given snapshot S and
    work queue W.  Returns an array indexed by W position (-2 elsewhere)."""
    S, W, ch = _i32(S), _i32(W), _i32(chunks)
    out = np.full(max(len(W), 1), -2, np.int32)
    rc = _load().orc_rs_chunks(*_g(g), _p(S), _p(W), len(W), policy, chunk, big_net,
                               _p(ch), len(ch), nthreads, _p(out))
    if rc != OK:
        raise ValueError(f"orc_rs_chunks failed: {rc}")
    return out[:len(W)]


def rs_losers(g, c, W, which):
    """Conflict rule of O-2 for the listed W positions -> (lose flags, status)."""
    c, W, wh = _i32(c), _i32(W), _i32(which)
    lose = np.zeros(max(len(wh), 1), np.uint8)
    rc = _load().orc_rs_losers(*_g(g), _p(c), _p(W), len(W), _p(wh), len(wh),
                               lose.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return lose[:len(wh)], rc


def conflicts(g, c) -> int:
    """V_A vertices that are uncolored or share a color with a two-hop neighbour."""
    return int(_load().orc_conflicts(*_g(g), _p(_i32(c))))


def max_nbor(g):
    """(max_w |nbor(w)|, per-vertex |nbor(w)|): the greedy bound's ingredients."""
    sizes = np.empty(max(g.n_a, 1), np.int32)
    best = _load().orc_max_nbor(*_g(g), _p(sizes))
    return int(best), sizes[:g.n_a]


def bruteforce_min(g) -> int:
    """Minimum number of colors of a valid BGPC coloring (n_a <= 20)."""
    k = _load().orc_bruteforce_min(*_g(g))
    if k < 0:
        raise ValueError("graph too large for exhaustive search")
    return int(k)


def closed_nbhd(ug):
    """D2GC as BGPC: nets(u) = vtxs(u) = N[u] = {u} u adj(u) (Section IV)."""
    n = int(ug.n)
    cptr = np.empty(n + 1, np.int32)
    cidx = np.empty(int(ug.idx.shape[0]) + n, np.int32)
    _load().orc_closed_nbhd(n, _p(ug.ptr), _p(ug.idx), _p(cptr), _p(cidx))
    return SimpleNamespace(n_a=n, n_b=n, a_ptr=cptr, a_idx=cidx, b_ptr=cptr, b_idx=cidx)


def d2_conflicts(ug, c) -> int:
    """Vertices uncolored or sharing a color within shortest-path distance 2."""
    return int(_load().orc_d2_conflicts(int(ug.n), _p(ug.ptr), _p(ug.idx), _p(_i32(c))))


def sl_rank(g):
    """Smallest-last order (Sec. VI, Tables II / IV) on the conflict graph:
    (rank, degeneracy); rank[w] = position of w in the coloring order."""
    rank = np.empty(max(g.n_a, 1), np.int32)
    dg = ctypes.c_int32(0)
    rc = _load().orc_sl_rank(*_g(g), _p(rank), ctypes.byref(dg))
    if rc != OK:
        raise ValueError(f"orc_sl_rank failed: {rc}")
    return rank[:g.n_a], dg.value


def color_sets(c):
    """(number of non-empty color sets, cardinality per color 0..max)."""
    c = _i32(c)
    mx = int(c.max()) if c.size else -1
    card = np.zeros(max(mx + 1, 1), np.int64)
    K = ctypes.c_int32(0)
    _load().orc_color_sets(len(c), _p(c), ctypes.byref(K), _p64(card))
    return K.value, card[:mx + 1]


def balance(c):
    """Table VI statistics: #color sets, max / mean / std of set cardinality."""
    K, card = color_sets(c)
    nz = card[card > 0].astype(np.float64)
    if nz.size == 0:
        return dict(colors=0, max_card=0, mean_card=0.0, std_card=0.0)
    return dict(colors=K, max_card=int(nz.max()), mean_card=float(nz.mean()),
                std_card=float(nz.std()))
