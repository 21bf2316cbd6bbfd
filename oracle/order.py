"""Oracle for the learned vertex order (plain numpy, float64).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``).

The paper colors vertices in a given order and discusses how the order
changes the number of colors (static orderings such as smallest-last, Sec. VI
and the related-work discussion of orderings).  The learned order replaces a
static ordering heuristic by a small regression model over per-vertex
statistics of the bipartite graph: the vertex's nets and their sizes, the
quantities the paper's cost analysis is written in (|nets(w)|, |vtxs(v)| and
the two-hop volume of Sec. III).

Everything here is the plain definition, evaluated in float64:

* ``features``: eight statistics per vertex of V_A, each passed through
  log1p (counts span many orders of magnitude on power-law graphs).
* ``bf16``: round-to-nearest-even of a float32 to the 8-bit-mantissa bfloat16
  format (IEEE 754 rounding, applied to the top 16 bits of the float32).
* ``forward`` / ``grad``: the MLP 8 -> 64 -> 64 -> 1 with ReLU, weights taken
  as their bfloat16 values, mean squared error loss; the gradient is the
  textbook backpropagation of that loss (straight through the weight
  rounding).
* ``adam``: one step of Adam (Kingma and Ba, 2015) with bias correction.
* ``rank_from_scores``: position of each vertex when the vertices are sorted
  by decreasing score, equal scores by increasing vertex id; -0.0 equals
  +0.0.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 8, 64
# packed parameter layout: W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3
OFF_W1, OFF_B1 = 0, 512
OFF_W2, OFF_B2 = 576, 4672
OFF_W3, OFF_B3 = 4736, 4800
N_PARAMS = 4801
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def features_of(g, vertices, big_net: int) -> np.ndarray:
    """Features (float64) of the listed vertices: for vertex w with net sizes
    s_v, v in nets(w): log1p of deg, mean s, max s, sum s, sum (s - 1),
    min s, #{s > T}, sum s^2 / sum s.  A vertex with no nets has all-zero
    features."""
    sizes = np.diff(np.asarray(g.b_ptr, np.int64)).astype(np.float64)
    a_ptr = np.asarray(g.a_ptr, np.int64)
    a_idx = np.asarray(g.a_idx, np.int64)
    X = np.zeros((len(vertices), N_IN))
    for r, w in enumerate(vertices):
        s = sizes[a_idx[a_ptr[w]:a_ptr[w + 1]]]
        if s.size == 0:
            continue
        tot = s.sum()
        raw = [s.size, tot / s.size, s.max(), tot, (s - 1).sum(), s.min(),
               float((s > big_net).sum()), (s * s).sum() / tot]
        X[r] = np.log1p(raw)
    return X


def features(g, big_net: int) -> np.ndarray:
    """X[n_a, 8] (float64): ``features_of`` every vertex of V_A."""
    return features_of(g, range(g.n_a), big_net)


def bf16(x32: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); the result
    is returned as float32 values.  Finite inputs only."""
    u = np.asarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def unpack(params: np.ndarray):
    p = np.asarray(params, np.float64)
    W1 = p[OFF_W1:OFF_B1].reshape(N_HID, N_IN)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(N_HID, N_HID)
    b2 = p[OFF_B2:OFF_W3]
    W3 = p[OFF_W3:OFF_B3]
    b3 = p[OFF_B3]
    return W1, b1, W2, b2, W3, b3


def forward(params_bf16: np.ndarray, X: np.ndarray):
    """Scores s[n] and the activations (z1, h1, z2, h2) for ``grad``."""
    W1, b1, W2, b2, W3, b3 = unpack(params_bf16)
    X = np.asarray(X, np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    s = h2 @ W3 + b3
    return s, (z1, h1, z2, h2)


def loss(params_bf16, X, y) -> float:
    s, _ = forward(params_bf16, X)
    return float(np.mean((s - np.asarray(y, np.float64)) ** 2))


def grad(params_bf16: np.ndarray, X: np.ndarray, y: np.ndarray):
    """(dL/dparams[4801], L) for L = mean (s - y)^2, by backpropagation."""
    W1, b1, W2, b2, W3, b3 = unpack(params_bf16)
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    n = X.shape[0]
    s, (z1, h1, z2, h2) = forward(params_bf16, X)
    ds = 2.0 * (s - y) / n
    g = np.zeros(N_PARAMS)
    g[OFF_W3:OFF_B3] = ds @ h2
    g[OFF_B3] = ds.sum()
    dz2 = np.outer(ds, W3) * (z2 > 0)
    g[OFF_W2:OFF_B2] = (dz2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g[OFF_W1:OFF_B1] = (dz1.T @ X).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    return g, float(np.mean((s - y) ** 2))


def adam(w, m, v, g, step: int, lr: float):
    """Adam step number ``step`` (1-based): returns new (w, m, v)."""
    w = np.asarray(w, np.float64)
    m = BETA1 * np.asarray(m, np.float64) + (1 - BETA1) * g
    v = BETA2 * np.asarray(v, np.float64) + (1 - BETA2) * g * g
    mh = m / (1 - BETA1 ** step)
    vh = v / (1 - BETA2 ** step)
    return w - lr * mh / (np.sqrt(vh) + EPS), m, v


def rank_from_scores(score32: np.ndarray) -> np.ndarray:
    """rank[w] = position of w in the order of decreasing score, ties by
    increasing w (scores compared as float32 values, -0.0 == +0.0)."""
    s = np.asarray(score32, np.float32)
    if np.isnan(s).any():
        raise ValueError("NaN score")
    key = -s.astype(np.float64)  # exact: float32 -> float64
    order = np.lexsort((np.arange(s.size), key))
    rank = np.empty(s.size, np.int32)
    rank[order] = np.arange(s.size, dtype=np.int32)
    return rank
