"""Seeded synthetic evolving-graph workloads (inputs only, no G-REST arithmetic).

This module is the one piece shared by the CUDA path's harness and the CPU
oracle's tests: it produces graphs and update batches, nothing else.  It holds
none of the method's arithmetic (no operators, projections or eigensolvers).

Workload shapes follow the paper's experiments (Sec. 5):
* stochastic block models as in the clustering study (Sec. 5.5: p_in = 0.05,
  nodes join random communities, 50 new nodes per step);
* power-law graphs standing in for the SNAP / Network Repository datasets of
  Table 2, which are not available here: Chung-Lu graphs with expected-degree
  weights w_i proportional to (i + i0)^(-1/(gamma-1));
* graph growth of 0.5-1% new nodes per step (Sec. 5.1, Scenario 1) attached
  by preferential attachment, plus uniform edge deletions (Sec. 2, K block
  with -1 entries).

Edges are undirected; an edge is stored once as the int64 key u*2^32 + v with
u < v.  A batch lists every undirected edge once.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SHIFT = np.int64(32)
LOW = np.int64((1 << 32) - 1)


@dataclass
class Batch:
    """One update Delta of Eq. (adj_update): S new nodes plus edge edits.

    New nodes take ids n .. n+S-1 (Sec. 2).  `ins_*` adds edges (+1 entries of
    K, and the G and C blocks); `del_*` removes edges (-1 entries of K);
    `del_nodes` tombstones old nodes (node removal, which the paper leaves to
    future work; see the library header for the reading used).
    """
    n_new: int
    ins_u: np.ndarray
    ins_v: np.ndarray
    del_u: np.ndarray
    del_v: np.ndarray
    del_nodes: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    ins_w: np.ndarray | None = None

    @property
    def n_ins(self):
        return int(self.ins_u.size)

    @property
    def n_del(self):
        return int(self.del_u.size)


def keys_of(u, v):
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    return (a << SHIFT) | b


def split_keys(keys):
    keys = np.asarray(keys, np.int64)
    return (keys >> SHIFT).astype(np.int32), (keys & LOW).astype(np.int32)


class EdgeSetGraph:
    """Host-side bookkeeping of the evolving graph used to draw valid batches."""

    def __init__(self, n, keys, weights=None):
        self.n = int(n)
        order = np.argsort(keys, kind="stable")
        self.keys = np.asarray(keys, np.int64)[order]
        self.w = None if weights is None else np.asarray(weights, np.float64)[order]
        self.live = np.ones(self.n, dtype=bool)

    def copy(self):
        g = EdgeSetGraph.__new__(EdgeSetGraph)
        g.n = self.n
        g.keys = self.keys.copy()
        g.w = None if self.w is None else self.w.copy()
        g.live = self.live.copy()
        return g

    @property
    def n_edges(self):
        return int(self.keys.size)

    def degrees(self):
        u, v = split_keys(self.keys)
        d = np.bincount(u, minlength=self.n) + np.bincount(v, minlength=self.n)
        return d.astype(np.int64)

    def has(self, keys):
        keys = np.asarray(keys, np.int64)
        pos = np.searchsorted(self.keys, keys)
        pos = np.minimum(pos, max(self.keys.size - 1, 0))
        if self.keys.size == 0:
            return np.zeros(keys.shape, bool)
        return self.keys[pos] == keys

    def csr(self):
        """Symmetric CSR (rowptr int64, col int32, val float64 or None), rows sorted."""
        u, v = split_keys(self.keys)
        rows = np.concatenate([u, v]).astype(np.int64)
        cols = np.concatenate([v, u]).astype(np.int64)
        order = np.lexsort((cols, rows))
        rows, cols = rows[order], cols[order]
        rowptr = np.zeros(self.n + 1, np.int64)
        np.cumsum(np.bincount(rows, minlength=self.n), out=rowptr[1:])
        val = None
        if self.w is not None:
            val = np.concatenate([self.w, self.w])[order]
        return rowptr, cols.astype(np.int32), val

    def apply(self, b: Batch):
        """Apply a batch (assumed valid) to the bookkeeping copy."""
        self.n += int(b.n_new)
        self.live = np.concatenate([self.live, np.ones(int(b.n_new), bool)])
        if b.del_u.size:
            dk = keys_of(b.del_u, b.del_v)
            keep = ~np.isin(self.keys, dk)
            self.keys = self.keys[keep]
            if self.w is not None:
                self.w = self.w[keep]
        if b.del_nodes.size:
            u, v = split_keys(self.keys)
            dead = np.zeros(self.n, bool)
            dead[b.del_nodes] = True
            keep = ~(dead[u] | dead[v])
            self.keys = self.keys[keep]
            if self.w is not None:
                self.w = self.w[keep]
            self.live[b.del_nodes] = False
        if b.ins_u.size:
            ik = keys_of(b.ins_u, b.ins_v)
            allk = np.concatenate([self.keys, ik])
            order = np.argsort(allk, kind="stable")
            self.keys = allk[order]
            if self.w is not None:
                iw = b.ins_w if b.ins_w is not None else np.ones(ik.size)
                self.w = np.concatenate([self.w, iw])[order]


# ---------------------------------------------------------------- samplers

def _sample_pairs_bernoulli(rng, n_pairs, p):
    """Indices of Bernoulli(p) successes among n_pairs trials, sorted."""
    if n_pairs <= 0 or p <= 0:
        return np.zeros(0, np.int64)
    cnt = rng.binomial(n_pairs, p)
    if cnt == 0:
        return np.zeros(0, np.int64)
    if n_pairs <= 4 * 10**7:
        return np.sort(rng.choice(n_pairs, size=cnt, replace=False)).astype(np.int64)
    got = np.unique(rng.integers(0, n_pairs, size=int(cnt * 1.1) + 16))
    while got.size < cnt:
        more = rng.integers(0, n_pairs, size=cnt - got.size + 16)
        got = np.unique(np.concatenate([got, more]))
    return np.sort(rng.choice(got, size=cnt, replace=False)).astype(np.int64)


def _sample_upper_pairs(rng, ids, p):
    """Bernoulli(p) edges among the unordered pairs of `ids` (no self pairs)."""
    m = ids.size
    npairs = m * (m - 1) // 2
    if npairs == 0 or p <= 0:
        return np.zeros(0, np.int64)
    cnt = int(rng.binomial(npairs, p))
    got = np.zeros(0, np.int64)
    while got.size < cnt:
        need = cnt - got.size
        r = rng.integers(0, m, size=2 * need + 16)
        c = rng.integers(0, m, size=2 * need + 16)
        ok = r < c
        k = np.unique(r[ok].astype(np.int64) * m + c[ok])
        k = np.setdiff1d(k, got)
        got = np.concatenate([got, rng.permutation(k)[:need]])
    r, c = got // m, got % m
    return keys_of(ids[r], ids[c])


def sbm_graph(n, n_comm, p_in, p_out, seed, equal_sizes=True):
    """SBM edges: blocks of equal size (or uniform labels), pairs i<j Bernoulli."""
    rng = np.random.default_rng(seed)
    if equal_sizes:
        labels = np.repeat(np.arange(n_comm), int(np.ceil(n / n_comm)))[:n]
    else:
        labels = rng.integers(0, n_comm, size=n)
    keys = []
    members = [np.flatnonzero(labels == c) for c in range(n_comm)]
    for a in range(n_comm):
        ia = members[a]
        for b in range(a, n_comm):
            ib = members[b]
            if a == b:
                m = ia.size
                keys.append(_sample_upper_pairs(rng, ia, p_in))
            else:
                npairs = ia.size * ib.size
                idx = _sample_pairs_bernoulli(rng, npairs, p_out)
                keys.append(keys_of(ia[idx // ib.size], ib[idx % ib.size]))
    keys = np.unique(np.concatenate(keys)) if keys else np.zeros(0, np.int64)
    return EdgeSetGraph(n, keys), labels


def _sorted_unique(a):
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.empty(a.size, bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def chung_lu_graph(n, gamma, mean_deg, seed, i0=None):
    """Chung-Lu power-law graph by ball dropping; self-loops and repeats removed."""
    rng = np.random.default_rng(seed)
    if i0 is None:
        i0 = max(1, int(n ** 0.1))
    w = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (gamma - 1.0))
    w *= mean_deg * n / w.sum()
    cap = np.sqrt(w.sum())
    w = np.minimum(w, cap)
    w *= mean_deg * n / w.sum()
    m = int(round(n * mean_deg / 2))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    keys = np.zeros(0, np.int64)
    target = m
    tries = 0
    while keys.size < target and tries < 8:
        need = target - keys.size
        draw = int(need * 1.05) + 64
        # endpoints ~ w: sorted uniforms make the search sequential; a random
        # permutation of sorted i.i.d. draws is again i.i.d.
        u = rng.permutation(np.searchsorted(cdf, np.sort(rng.random(draw)), side="right"))
        v = rng.permutation(np.searchsorted(cdf, np.sort(rng.random(draw)), side="right"))
        u = np.minimum(u, n - 1)
        v = np.minimum(v, n - 1)
        ok = u != v
        keys = _sorted_unique(np.concatenate([keys, keys_of(u[ok], v[ok])]))
        tries += 1
    if keys.size > target:
        keys = np.sort(rng.choice(keys, size=target, replace=False))
    return EdgeSetGraph(n, keys)


def largest_component(g: EdgeSetGraph):
    """Relabel to the largest connected component (ids kept in original order)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    u, v = split_keys(g.keys)
    a = sp.coo_matrix((np.ones(u.size), (u, v)), shape=(g.n, g.n)).tocsr()
    ncomp, lab = connected_components(a, directed=False)
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    remap = -np.ones(g.n, np.int64)
    remap[keep] = np.arange(keep.size)
    ok = (remap[u] >= 0) & (remap[v] >= 0)
    return EdgeSetGraph(keep.size, keys_of(remap[u[ok]], remap[v[ok]]))


# ---------------------------------------------------------------- streams

def sbm_growth_batch(g: EdgeSetGraph, labels, n_comm, p_in, p_out, n_new, n_rand_edges, rng):
    """S new nodes join uniform communities with SBM edges to every current
    node (old and new), plus uniform new edges among non-adjacent old pairs."""
    n = g.n
    new_lab = rng.integers(0, n_comm, size=n_new)
    all_lab = np.concatenate([labels, new_lab])
    ins = []
    live_old = np.flatnonzero(g.live)
    for s in range(n_new):
        j = n + s
        cand = np.concatenate([live_old, np.arange(n, j)])
        p = np.where(all_lab[cand] == new_lab[s], p_in, p_out)
        hit = cand[rng.random(cand.size) < p]
        ins.append(keys_of(np.full(hit.size, j), hit))
    # uniform random edges among old, non-adjacent pairs
    extra = np.zeros(0, np.int64)
    while extra.size < n_rand_edges:
        need = n_rand_edges - extra.size
        u = rng.choice(live_old, size=2 * need + 8)
        v = rng.choice(live_old, size=2 * need + 8)
        ok = u != v
        k = keys_of(u[ok], v[ok])
        k = k[~g.has(k)]
        k = np.setdiff1d(np.unique(k), extra)
        extra = np.concatenate([extra, rng.permutation(k)[:need]])
    ins.append(extra[:n_rand_edges])
    ik = np.concatenate(ins)
    iu, iv = split_keys(ik)
    b = Batch(n_new=n_new, ins_u=iu, ins_v=iv, del_u=np.zeros(0, np.int32), del_v=np.zeros(0, np.int32))
    return b, all_lab


def pa_growth_batch(g: EdgeSetGraph, n_new, edges_per_node, n_delete, rng, new_new_frac=0.0):
    """S new nodes attach `edges_per_node` distinct degree-proportional old
    targets each; `n_delete` existing edges are removed uniformly at random."""
    n = g.n
    deg = g.degrees().astype(np.float64)
    deg[~g.live] = 0.0
    wsum = deg.sum()
    cdf = np.cumsum(deg) / wsum
    ins = []
    for s in range(n_new):
        j = n + s
        t = np.zeros(0, np.int64)
        while t.size < edges_per_node:
            d = np.searchsorted(cdf, rng.random(2 * edges_per_node), side="right")
            d = np.minimum(d, n - 1)
            t = np.unique(np.concatenate([t, d[deg[d] > 0]]))
        t = rng.permutation(t)[:edges_per_node]
        ins.append(keys_of(np.full(t.size, j), t))
    ik = np.concatenate(ins) if ins else np.zeros(0, np.int64)
    if new_new_frac > 0 and n_new > 1:
        nn = int(new_new_frac * n_new * edges_per_node)
        a = rng.integers(n, n + n_new, size=2 * nn + 4)
        b = rng.integers(n, n + n_new, size=2 * nn + 4)
        ok = a != b
        k = np.setdiff1d(np.unique(keys_of(a[ok], b[ok])), ik)[:nn]
        ik = np.concatenate([ik, k])
    dk = np.zeros(0, np.int64)
    if n_delete > 0 and g.n_edges:
        dk = np.sort(rng.choice(g.keys, size=min(n_delete, g.n_edges), replace=False))
    iu, iv = split_keys(ik)
    du, dv = split_keys(dk)
    return Batch(n_new=n_new, ins_u=iu, ins_v=iv, del_u=du, del_v=dv)


def random_churn_batch(g: EdgeSetGraph, n_new, n_ins, n_del, rng, n_del_nodes=0, new_edges_per_node=3):
    """Generic valid batch: new nodes with a few random edges, random inserts
    among non-adjacent live pairs, random deletions, optional node deletions."""
    n = g.n
    live = np.flatnonzero(g.live)
    del_nodes = np.zeros(0, np.int32)
    if n_del_nodes:
        del_nodes = np.sort(rng.choice(live, size=n_del_nodes, replace=False)).astype(np.int32)
    dead = np.zeros(n, bool)
    dead[del_nodes] = True
    alive = live[~dead[live]]
    # deletions among edges not touching deleted nodes
    u, v = split_keys(g.keys)
    cand = g.keys[~(dead[u] | dead[v])]
    dk = np.sort(rng.choice(cand, size=min(n_del, cand.size), replace=False)) if n_del and cand.size else np.zeros(0, np.int64)
    ins = np.zeros(0, np.int64)
    while ins.size < n_ins:
        need = n_ins - ins.size
        a = rng.choice(alive, size=2 * need + 8)
        b = rng.choice(alive, size=2 * need + 8)
        ok = a != b
        k = np.unique(keys_of(a[ok], b[ok]))
        k = k[~g.has(k)]
        k = np.setdiff1d(k, ins)
        ins = np.concatenate([ins, rng.permutation(k)[:need]])
    newk = []
    for s in range(n_new):
        j = n + s
        t = rng.choice(alive, size=min(new_edges_per_node, alive.size), replace=False)
        newk.append(keys_of(np.full(t.size, j), t))
        if s > 0 and rng.random() < 0.5:
            newk.append(keys_of([j], [n + rng.integers(0, s)]))
    ik = np.concatenate([ins] + newk) if newk else ins
    ik = np.unique(ik)
    iu, iv = split_keys(rng.permutation(ik))
    du, dv = split_keys(dk)
    return Batch(n_new=n_new, ins_u=iu, ins_v=iv, del_u=du, del_v=dv, del_nodes=del_nodes)


# ---------------------------------------------------------------- configs

def sbm_stream(seed=20260304, n0=2000, n_comm=4, p_in=0.05, p_out=0.005, steps=10, n_new=50, n_rand=200):
    """SBM n=2,000, 4 equal communities, 10 steps of +50 nodes and +200 edges."""
    g, lab = sbm_graph(n0, n_comm, p_in, p_out, seed)
    g0 = g.copy()
    rng = np.random.default_rng(seed + 1)
    batches = []
    for _ in range(steps):
        b, lab = sbm_growth_batch(g, lab, n_comm, p_in, p_out, n_new, n_rand, rng)
        g.apply(b)
        batches.append(b)
    return g0, batches


def chung_lu_stream(n, gamma, mean_deg, steps, grow_frac, edges_per_node, del_frac, seed, lcc=False):
    """Power-law stream: +grow_frac*N nodes by preferential attachment and
    -del_frac*|E| uniform deletions per step."""
    g = chung_lu_graph(n, gamma, mean_deg, seed)
    if lcc:
        g = largest_component(g)
    g0 = g.copy()
    rng = np.random.default_rng(seed + 1)
    batches = []
    for _ in range(steps):
        S = int(np.floor(grow_frac * g.n))
        nd = int(np.floor(del_frac * g.n_edges))
        b = pa_growth_batch(g, S, edges_per_node, nd, rng)
        g.apply(b)
        batches.append(b)
    return g0, batches


class PowerLawStream:
    """Fast generator of the power-law growth stream: per step, S new nodes
    attach `edges_per_node` distinct old targets drawn proportionally to degree
    (preferential attachment) and `n_delete` uniformly chosen existing edges
    are removed.  Edges live in an append-only key array with an alive mask,
    so no step needs a search over the whole edge set."""

    def __init__(self, g: EdgeSetGraph, seed):
        self.rng = np.random.default_rng(seed)
        self.n = g.n
        self.keys = g.keys.copy()
        self.alive = np.ones(self.keys.size, bool)
        self.n_alive = int(self.keys.size)
        self.deg = g.degrees().astype(np.float64)

    def next_batch(self, S, edges_per_node, n_delete):
        rng = self.rng
        n = self.n
        cdf = np.cumsum(self.deg[:n])
        cdf /= cdf[-1]
        c = 3 * edges_per_node
        cand = np.searchsorted(cdf, rng.random((S, c)), side="right")
        np.minimum(cand, n - 1, out=cand)
        # first occurrences per row in draw order, keep the first edges_per_node
        order = np.argsort(cand, axis=1, kind="stable")
        srt = np.take_along_axis(cand, order, axis=1)
        dup_s = np.zeros_like(srt, dtype=bool)
        dup_s[:, 1:] = srt[:, 1:] == srt[:, :-1]
        dup = np.zeros_like(dup_s)
        np.put_along_axis(dup, order, dup_s, axis=1)
        rank = np.cumsum(~dup, axis=1)
        keep = (~dup) & (rank <= edges_per_node)
        rows, cols = np.nonzero(keep)
        tgt = cand[rows, cols].astype(np.int64)
        newid = (n + rows).astype(np.int64)
        ik = keys_of(tgt, newid)
        # uniform deletions among alive edges
        dk = np.zeros(0, np.int64)
        if n_delete > 0:
            alive_idx = np.flatnonzero(self.alive)
            pick = rng.choice(alive_idx.size, size=min(n_delete, alive_idx.size), replace=False)
            di = np.sort(alive_idx[pick])
            dk = self.keys[di]
            self.alive[di] = False
            du, dv = split_keys(dk)
            np.subtract.at(self.deg, du, 1.0)
            np.subtract.at(self.deg, dv, 1.0)
        # commit the insertions
        self.deg = np.concatenate([self.deg, np.zeros(S)])
        np.add.at(self.deg, tgt, 1.0)
        np.add.at(self.deg, newid, 1.0)
        self.keys = np.concatenate([self.keys, ik])
        self.alive = np.concatenate([self.alive, np.ones(ik.size, bool)])
        self.n = n + S
        iu, iv = split_keys(ik)
        du, dv = split_keys(dk)
        return Batch(n_new=S, ins_u=iu, ins_v=iv, del_u=du, del_v=dv)


def power_law_workload(n, gamma, mean_deg, steps, grow_frac, edges_per_node, del_frac, seed, lcc=False):
    """Initial Chung-Lu graph and `steps` batches of the growth stream
    (+grow_frac*N nodes, -del_frac*|E| edges per step), sizes taken from the
    graph at the start of each step."""
    g = chung_lu_graph(n, gamma, mean_deg, seed)
    if lcc:
        g = largest_component(g)
    st = PowerLawStream(g, seed + 1)
    batches = []
    for _ in range(steps):
        S = int(np.floor(grow_frac * st.n))
        nd = int(np.floor(del_frac * st.n_alive))
        b = st.next_batch(S, edges_per_node, nd)
        st.n_alive += b.n_ins - b.n_del
        batches.append(b)
    return g, batches


def csr_fast(g: EdgeSetGraph):
    """Symmetric CSR of an EdgeSetGraph without per-row column sorting."""
    u, v = split_keys(g.keys)
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    order = np.argsort(rows, kind="stable")
    rowptr = np.zeros(g.n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=g.n), out=rowptr[1:])
    val = None if g.w is None else np.concatenate([g.w, g.w])[order]
    return rowptr, cols[order].astype(np.int32), val
