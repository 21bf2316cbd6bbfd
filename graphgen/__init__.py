"""Seeded synthetic inputs for the BGPC / D2GC workloads.

This package only builds graphs (int32 CSR over V_A plus CSC over V_B, both
sorted and duplicate-free).  It holds none of the coloring method's arithmetic
and is the one module that the CPU oracle's tests, the GPU tests and the
benchmark all share.  The generators live in ``graphgen.c`` (counter-based
SplitMix64 stream, so a graph depends only on its parameters and seed).

Workload recipes (the stand-ins for the paper's UFL / MovieLens matrices of
Table II, which are not available here):

* ``random_bipartite(2000, 2000, 5, seed=1)``: small uniform case.
* ``stencil9(1024)``: Jacobian pattern of a 2D 9-point stencil, standing in
  for the PDE matrices (af_shell, bone010, channel, nlpkkt120).
* ``chung_lu(1 << 22, 16, 50000, 2.1, seed)``: skewed power-law bipartite
  graph, standing in for coPapersDBLP / uk-2002 / 20M_movielens.
* ``rmat(22, 16, .57, .19, .19, seed)``: undirected R-MAT graph for D2GC.
* ``batch_graph(seed, i)``: graph ``i`` of the 512-graph batched workload.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_build", "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (no-op when up to date)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i32, i64, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_uint64, ctypes.c_double)
        P = ctypes.POINTER(ctypes.c_int32)
        for name, args in {
            "gg_random_bipartite": [i32, i32, i32, u64],
            "gg_stencil9": [i32],
            "gg_chung_lu": [i32, dbl, dbl, dbl, u64],
            "gg_rmat": [i32, i32, dbl, dbl, dbl, u64],
            "gg_from_edges": [i32, i64, P, P],
            "gg_from_pairs": [i32, i32, i64, P, P],
            "gg_batch_graph": [u64, i32, dbl, dbl, dbl, i32],
        }.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = vp
        lib.gg_batch_sizes.argtypes = [u64, i32, dbl, dbl, P, P]
        lib.gg_batch_sizes.restype = None
        for name in ("gg_n_a", "gg_n_b", "gg_nnz"):
            getattr(lib, name).argtypes = [vp]
            getattr(lib, name).restype = i64
        lib.gg_undirected.argtypes = [vp]
        lib.gg_undirected.restype = ctypes.c_int
        lib.gg_copy.argtypes = [vp, P, P, P, P]
        lib.gg_copy.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_free.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


@dataclass
class BGraph:
    """Bipartite graph G = (V_A u V_B, E): nets(u) = a_idx[a_ptr[u]:a_ptr[u+1]],
    vtxs(v) = b_idx[b_ptr[v]:b_ptr[v+1]] (int32, sorted, unique)."""
    n_a: int
    n_b: int
    a_ptr: np.ndarray
    a_idx: np.ndarray
    b_ptr: np.ndarray
    b_idx: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.a_idx.shape[0])


@dataclass
class UGraph:
    """Undirected graph without self loops: adj(u) = idx[ptr[u]:ptr[u+1]]."""
    n: int
    ptr: np.ndarray
    idx: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])


def _take(h, name: str, undirected: bool):
    lib = _load()
    try:
        n_a, n_b, nnz = lib.gg_n_a(h), lib.gg_n_b(h), lib.gg_nnz(h)
        a_ptr = np.empty(n_a + 1, np.int32)
        a_idx = np.empty(nnz, np.int32)
        if undirected:
            lib.gg_copy(h, _p(a_ptr), _p(a_idx), None, None)
            return UGraph(int(n_a), a_ptr, a_idx, name)
        b_ptr = np.empty(n_b + 1, np.int32)
        b_idx = np.empty(nnz, np.int32)
        lib.gg_copy(h, _p(a_ptr), _p(a_idx), _p(b_ptr), _p(b_idx))
        return BGraph(int(n_a), int(n_b), a_ptr, a_idx, b_ptr, b_idx, name)
    finally:
        lib.gg_free(h)


def random_bipartite(n_a: int, n_b: int, deg: int, seed: int = 1) -> BGraph:
    """Each V_A vertex joins `deg` distinct V_B nets drawn uniformly."""
    return _take(_load().gg_random_bipartite(n_a, n_b, deg, seed),
                 f"random_{n_a}x{n_b}_d{deg}_s{seed}", False)


def stencil9(n: int) -> BGraph:
    """Jacobian sparsity of a 9-point stencil on an n x n grid (row-major ids)."""
    return _take(_load().gg_stencil9(n), f"stencil9_{n}x{n}", False)


def chung_lu(n: int, mean: float = 16.0, wmax: float = 50000.0, beta: float = 2.1,
             seed: int = 2) -> BGraph:
    """Power-law (Chung-Lu) bipartite graph with n vertices on each side."""
    return _take(_load().gg_chung_lu(n, mean, wmax, beta, seed),
                 f"chung_lu_{n}_m{mean:g}_w{wmax:g}_b{beta:g}_s{seed}", False)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 3) -> UGraph:
    """Undirected R-MAT graph (symmetrised, deduplicated, no self loops)."""
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, seed),
                 f"rmat_s{scale}_ef{edge_factor}_s{seed}", True)


def from_edges(n: int, edges) -> UGraph:
    """Undirected graph from an edge list (symmetrised, deduplicated)."""
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    s, d = np.ascontiguousarray(e[:, 0]), np.ascontiguousarray(e[:, 1])
    return _take(_load().gg_from_edges(n, len(e), _p(s), _p(d)), "edges", True)


def from_pairs(n_a: int, n_b: int, pairs) -> BGraph:
    """Bipartite graph from (u in V_A, v in V_B) incidences (deduplicated)."""
    e = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
    u, v = np.ascontiguousarray(e[:, 0]), np.ascontiguousarray(e[:, 1])
    return _take(_load().gg_from_pairs(n_a, n_b, len(e), _p(u), _p(v)), "pairs", False)


def from_nets(n_a: int, nets) -> BGraph:
    """Bipartite graph whose net v holds the V_A vertices listed in nets[v]."""
    pairs = [(u, v) for v, members in enumerate(nets) for u in members]
    if not pairs:
        z = np.zeros(0, np.int32)
        return BGraph(n_a, len(nets), np.zeros(n_a + 1, np.int32), z,
                      np.zeros(len(nets) + 1, np.int32), z.copy(), "nets")
    return from_pairs(n_a, len(nets), pairs)


def batch_sizes(seed: int, index: int, lo: float = 1e3, hi: float = 1e6):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _load().gg_batch_sizes(seed, index, lo, hi, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def batch_graph(seed: int, index: int, lo: float = 1e3, hi: float = 1e6,
                lam: float = 8.0, maxdeg: int = 64) -> BGraph:
    """Graph `index` of the batched workload: |V_A| log-uniform in [lo, hi],
    |V_B| = |V_A| * U[0.5, 2], degree Poisson(lam) clipped to [1, maxdeg]."""
    return _take(_load().gg_batch_graph(seed, index, lo, hi, lam, maxdeg),
                 f"batch_s{seed}_{index}", False)



def mlp_init(seed: int):
    """Initial parameters [4801] (float32) of the order model 8 -> 64 -> 64 -> 1,
    packed W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3: every weight and
    bias of a layer with fan-in f drawn uniform in [-1/sqrt(f), 1/sqrt(f)]
    (numpy PCG64 stream of ``seed``)."""
    rng = np.random.default_rng([0x6d6c70, seed])
    parts = []
    for fan_in, count in ((8, 64 * 8 + 64), (64, 64 * 64 + 64), (64, 64 + 1)):
        b = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-b, b, count))
    return np.concatenate(parts).astype(np.float32)
