"""DBSCAN on fixed-radius neighbour lists (Section 6.4), CPU oracle.

Test infrastructure (see the package docstring).  The paper runs
scikit-learn's DBSCAN with SNN as its neighbour search (Section 6.4); the
semantics are read as follows (the paper is silent on tie rules):

* N_eps(i) = brute-force neighbours of i with S <= eps^2, i itself included;
* core iff |N_eps(i)| >= minPts;
* clusters = connected components of the graph whose vertices are the core
  points and whose edges join core points that are neighbours;
* a non-core point with at least one core neighbour (a border point) joins the
  cluster of its smallest-id core neighbour (scikit-learn's choice depends on
  visiting order; this rule makes the labelling unique);
* a cluster's label is the smallest id among its members (cores and borders);
  every other point is noise, label -1.
"""
from __future__ import annotations

from collections import deque

import numpy as np
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

from .brute import brute_radius, CSR


def dbscan(P: np.ndarray, eps: float, min_pts: int, csr: CSR | None = None):
    """Returns (labels int32 n, is_core uint8 n)."""
    csr = brute_radius(P, None, eps) if csr is None else csr
    n = csr.m
    counts = csr.counts()
    core = counts >= min_pts
    rows = np.repeat(np.arange(n), counts)
    cols = csr.ids.astype(np.int64)
    cc = core[rows] & core[cols]
    g = csr_matrix((np.ones(int(cc.sum()), dtype=np.int8), (rows[cc], cols[cc])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    # border: smallest-id core neighbour (ids are ascending within a row)
    assign = np.full(n, -1, dtype=np.int64)
    assign[core] = comp[core]
    border_edges = (~core[rows]) & core[cols]
    br, bc = rows[border_edges], cols[border_edges]
    first = np.ones(len(br), dtype=bool)
    first[1:] = br[1:] != br[:-1]
    assign[br[first]] = comp[bc[first]]
    labels = np.full(n, -1, dtype=np.int64)
    member = assign >= 0
    if member.any():
        ncomp = int(comp.max()) + 1
        minid = np.full(ncomp, np.iinfo(np.int64).max, dtype=np.int64)
        np.minimum.at(minid, assign[member], np.nonzero(member)[0])
        labels[member] = minid[assign[member]]
    return labels.astype(np.int32), core.astype(np.uint8)


def dbscan_bfs(P: np.ndarray, eps: float, min_pts: int, csr: CSR | None = None):
    """Independent restatement by breadth-first expansion from each unvisited
    core point in ascending id order (small inputs).  Same semantics."""
    csr = brute_radius(P, None, eps) if csr is None else csr
    n = csr.m
    nb = [csr.row(i)[0] for i in range(n)]
    core = np.array([len(nb[i]) >= min_pts for i in range(n)])
    cluster = np.full(n, -1, dtype=np.int64)
    nclus = 0
    for s in range(n):
        if not core[s] or cluster[s] >= 0:
            continue
        cluster[s] = nclus
        dq = deque([s])
        while dq:
            i = dq.popleft()
            for j in nb[i]:
                if core[j] and cluster[j] < 0:
                    cluster[j] = nclus
                    dq.append(j)
        nclus += 1
    labels = np.full(n, -1, dtype=np.int64)
    owner = cluster.copy()
    for i in range(n):
        if core[i]:
            continue
        cores = [j for j in nb[i] if core[j]]
        if cores:
            owner[i] = cluster[min(cores)]
    for c in range(nclus):
        members = np.nonzero(owner == c)[0]
        labels[members] = members.min()
    return labels.astype(np.int32), core.astype(np.uint8)
