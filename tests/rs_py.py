"""A second, independent statement of the round-synchronous semantics in plain
Python sets, for tiny graphs only.  Used to cross-check the C oracle
(written separately, in C, with stamp arrays) on many small random cases.

Semantics (Alg. 1-4 and 8 of Tas, Kaya, Saule, rendered round-synchronously):
see oracle/bgpc_oracle.c, "O-2".
"""


def wave_of(j, Q):
    """Wave of chunk j: floor(frac(j * phi) * Q) in 32-bit fixed point."""
    x = (j * 0x9E3779B9) % (1 << 32)
    return (x * Q) >> 32


def nbors(nets_of, vtxs_of, w):
    out = set()
    for v in nets_of[w]:
        out.update(vtxs_of[v])
    out.discard(w)
    return out


def policy(pol, F, w, state):
    if pol == 1:  # B1
        if w % 2 == 0:
            col = state["col_max"]
            while col >= 0 and col in F:
                col -= 1
            if col == -1:
                col = state["col_max"] + 1
                while col in F:
                    col += 1
            return col
        col = 0
        while col in F:
            col += 1
        return col
    if pol in (2, 3):  # B2 / B2X
        col = state["col_next"]
        while col in F:
            col += 1
        if col > state["col_max"]:
            col = 0
            while col in F:
                col += 1
        return col
    col = 0
    while col in F:
        col += 1
    return col


def update(pol, col, state):
    state["col_max"] = max(state["col_max"], col)
    if pol == 2:
        state["col_next"] = min(col + 1, state["col_max"] // 3 + 1)
    elif pol == 3:
        state["col_next"] = max(col + 1, state["col_max"] // 3 + 1)


def rs(n_a, nets, pol=0, C=64, Q=16, T=64, rank=None, max_rounds=10_000, net_rounds=0,
       center_first=False):
    """nets: list of member lists (vtxs).  Returns (colors, w_per_round).
    The first net_rounds rounds are net-based (Alg. 8 / Alg. 9): each net
    proposes reverse first-fit colors to its uncolored members, read from the
    round's snapshot, and each vertex keeps its owner net's proposal."""
    vtxs_of = [sorted(set(m)) for m in nets]
    nets_of = [[] for _ in range(n_a)]
    for v, mem in enumerate(vtxs_of):
        for u in mem:
            nets_of[u].append(v)
    nb = [nbors(nets_of, vtxs_of, w) for w in range(n_a)]
    own = {}
    for w in range(n_a):
        best = None
        for v in nets_of[w]:
            key = (len(vtxs_of[v]), v)
            if best is None or key > best:
                best = key
        own[w] = best[1] if best else None
    size_own = {w: (len(vtxs_of[own[w]]) if own[w] is not None else 0) for w in range(n_a)}

    order = sorted(range(n_a), key=lambda w: (rank[w] if rank is not None else w))
    c = [-1] * n_a
    W = list(order)
    hist = []
    while W:
        if len(hist) >= max_rounds:
            raise RuntimeError("round cap")
        hist.append(len(W))
        pos = {w: p for p, w in enumerate(W)}
        k = {}
        for v, mem in enumerate(vtxs_of):
            if len(mem) <= T:
                continue
            cnt = 0
            for u in mem:
                if u in pos and own[u] == v:
                    k[u] = cnt
                    cnt += 1
        S = list(c)
        m = len(W)
        nch = (m + C - 1) // C
        net_round = len(hist) <= net_rounds
        if net_round:
            for v, mem in enumerate(vtxs_of):
                visit = list(mem)
                if center_first and v in visit:
                    visit.remove(v)
                    visit.insert(0, v)
                F, todo = set(), []
                for u in visit:
                    if S[u] != -1 and S[u] not in F:
                        F.add(S[u])
                    else:
                        todo.append(u)
                free = [x for x in range(len(mem) - 1, -1, -1) if x not in F]
                for i, u in enumerate(todo):
                    if own[u] == v and u in pos:
                        c[u] = free[i]
        for q in range(0 if net_round else Q):
            staged = {}
            for j in [j for j in range(nch) if wave_of(j, Q) == q]:
                L = {}
                st = {"col_max": max(max(S), 0) if S else 0, "col_next": 0}
                for w in W[j * C:(j + 1) * C]:
                    F = set()
                    for u in nb[w]:
                        cu = L[u] if u in L else S[u]
                        if cu >= 0:
                            F.add(cu)
                    col = -1
                    if size_own[w] > T:
                        free = [x for x in range(size_own[w] - 1, -1, -1) if x not in F]
                        if k[w] < len(free):
                            col = free[k[w]]
                    if col < 0:
                        col = policy(pol, F, w, st)
                    update(pol, col, st)
                    L[w] = col
                    staged[w] = col
            for w, col in staged.items():
                S[w] = col
        if not net_round:
            c = S
        losers = []
        for p, w in enumerate(W):
            lose = c[w] < 0
            for u in nb[w]:
                if c[u] == c[w] and c[w] >= 0:
                    assert net_round or u in pos, "a W vertex took a fixed neighbour's color"
                    if u not in pos or pos[u] < p:
                        lose = True
            if lose:
                losers.append(w)
        for w in losers:
            c[w] = -1
        W = losers
    return c, hist


def seq(n_a, nets, pol=0, rank=None):
    """Sequential greedy (one thread, Alg. 1 + Alg. 4 gather), direct loop."""
    vtxs_of = [sorted(set(m)) for m in nets]
    nets_of = [[] for _ in range(n_a)]
    for v, mem in enumerate(vtxs_of):
        for u in mem:
            nets_of[u].append(v)
    order = sorted(range(n_a), key=lambda w: (rank[w] if rank is not None else w))
    c = [-1] * n_a
    st = {"col_max": 0, "col_next": 0}
    for w in order:
        F = {c[u] for u in nbors(nets_of, vtxs_of, w) if c[u] >= 0}
        col = policy(pol, F, w, st)
        update(pol, col, st)
        c[w] = col
    return c
