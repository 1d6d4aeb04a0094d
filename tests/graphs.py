"""Small graph constructors shared by the tests (input construction only)."""
import numpy as np


def directed_csr(n_vertices, src, dst, offsets=np.int64):
    """CSR holding exactly the given arcs (no symmetrisation), rows in input order."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int32)
    order = np.argsort(src, kind="stable")
    counts = np.bincount(src, minlength=n_vertices) if src.size else np.zeros(n_vertices, np.int64)
    row_ptr = np.zeros(n_vertices + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr.astype(offsets), np.ascontiguousarray(dst[order], np.int32)


def symmetric_csr(n_vertices, src, dst, offsets=np.int64):
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    return directed_csr(n_vertices, np.concatenate([src, dst]), np.concatenate([dst, src]), offsets)


def path_edges(order):
    order = np.asarray(order, np.int64)
    return order[:-1], order[1:]


def clique_edges(members):
    members = list(members)
    s, d = [], []
    for i in range(len(members)):
        for j in range(i + 1, len(members)):
            s.append(members[i])
            d.append(members[j])
    return np.array(s, np.int64), np.array(d, np.int64)


def grid_edges(side, keep=None):
    """All lattice edges of a side x side grid with row-major IDs (keep: optional bool mask)."""
    s, d = [], []
    for r in range(side):
        for c in range(side):
            v = r * side + c
            if c + 1 < side:
                s.append(v); d.append(v + 1)
            if r + 1 < side:
                s.append(v); d.append(v + side)
    s, d = np.array(s, np.int64), np.array(d, np.int64)
    if keep is not None:
        s, d = s[keep], d[keep]
    return s, d


def closure_labels(n_vertices, src, dst):
    """Brute force: boolean reachability by Floyd-Warshall closure; label = min reachable vertex."""
    reach = np.eye(n_vertices, dtype=bool)
    for u, v in zip(src, dst):
        reach[u, v] = True
        reach[v, u] = True
    for k in range(n_vertices):
        reach |= reach[:, k:k + 1] & reach[k:k + 1, :]
    return np.array([int(np.argmax(reach[v])) for v in range(n_vertices)], np.int32)


def min_id_from_component_ids(comp):
    """Canonicalise arbitrary component IDs to the minimum vertex ID of each component."""
    comp = np.asarray(comp, np.int64)
    n = comp.shape[0]
    first = np.full(comp.max() + 1 if n else 0, np.iinfo(np.int64).max, np.int64)
    np.minimum.at(first, comp, np.arange(n, dtype=np.int64))
    return first[comp].astype(np.int32)


def check_min_label_invariants(row_ptr, col, labels):
    """Properties every correct min-ID labelling has; returns a list of violated ones."""
    labels = np.asarray(labels, np.int64)
    V = labels.shape[0]
    bad = []
    if V == 0:
        return bad
    if labels.min() < 0 or (labels > np.arange(V)).any():
        bad.append("label[v] <= v")
    if (labels[labels] != labels).any():
        bad.append("label[label[v]] == label[v]")
    rp = np.asarray(row_ptr, np.int64)
    src = np.repeat(np.arange(V, dtype=np.int64), np.diff(rp))
    if (labels[src] != labels[np.asarray(col, np.int64)]).any():
        bad.append("label[u] == label[v] on every arc")
    return bad
