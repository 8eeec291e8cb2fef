"""Blocked tall-skinny QR (TSQR), binary tree scheme, FP64.  Test infrastructure.

Sec. 3.3: partition K_hat into row blocks K_i, factor each K_i = Q_i R_i (Eq. 1), then
factor stacked pairs of R's (Eq. 2), and so on up the tree until one R remains (Eq. 3);
K_hat = (Q^b_1 Q^b_2 Q^b_3) R^b_3 (Eq. 4).  Readings:
  * leaves hold b rows each, in order; a last block with fewer than d rows is merged
    into its predecessor;
  * pairs are formed left to right at every level and an odd last node passes up
    unchanged;
  * each combine is a plain Householder QR of the stacked 2d x d matrix [R_a; R_b];
  * the final R is normalised to diag(R) >= 0 and Q_hat gets the matching column signs.
The block count the paper recommends, b = floor(n / 2r) + 1 (Sec. 3.3), disagrees with
its own four-block example (n = 8r, blocks of 2r rows); the leaf height is therefore a
parameter here.
"""
import numpy as np

from .householder import householder_qr, thin_q, normalise


def leaf_ranges(n, d, b):
    """Row ranges [start, stop) of the leaves."""
    if b < d or n < d:
        raise ValueError("need n >= d and block rows >= d")
    ranges = [(s, min(n, s + b)) for s in range(0, n, b)]
    if len(ranges) > 1 and ranges[-1][1] - ranges[-1][0] < d:
        s_prev = ranges[-2][0]
        ranges = ranges[:-2] + [(s_prev, n)]
    return ranges


def tsqr(Y, b, leaf_dtype=np.float64):
    """TSQR of the n x d matrix Y with leaves of b rows.

    Returns a dict with 'R' (d x d, diag >= 0), 'Q' (explicit thin Q_hat, n x d),
    'leaves' and 'levels' (the tree, for inspection).  `leaf_dtype` is the working
    precision of the leaf factorisations and of the leaves' part of Q_hat (float32 gives
    the floor of a method with FP32 leaves and an FP64 tree); the tree is always FP64."""
    Y = np.asarray(Y, dtype=np.float64)
    n, d = Y.shape
    ranges = leaf_ranges(n, d, b)
    leaves = []
    for (s, e) in ranges:
        V, tau, R = householder_qr(Y[s:e], leaf_dtype)
        leaves.append({"range": (s, e), "V": V, "tau": tau, "R": R.astype(np.float64)})
    # tree nodes: ('leaf', i) or ('node', a, b, V, tau); each carries its R
    level = [{"kind": "leaf", "index": i, "R": lf["R"]} for i, lf in enumerate(leaves)]
    levels = [level]
    while len(level) > 1:
        nxt = []
        for i in range(0, len(level) - 1, 2):
            a, c = level[i], level[i + 1]
            V, tau, R = householder_qr(np.vstack([a["R"], c["R"]]))
            nxt.append({"kind": "node", "children": (a, c), "V": V, "tau": tau, "R": R})
        if len(level) % 2 == 1:
            nxt.append(level[-1])
        level = nxt
        levels.append(level)
    root = level[0]

    def stacked_q(node):
        # Q of the subtree: stacked leaf R's = Q_sub R_node
        if node["kind"] == "leaf":
            return np.eye(d)
        a, c = node["children"]
        H = thin_q(node["V"], node["tau"])            # 2d x d
        Qa, Qc = stacked_q(a), stacked_q(c)
        return np.vstack([Qa @ H[:d], Qc @ H[d:]])

    Qtree = stacked_q(root)                             # (L d) x d
    Q = np.empty((n, d))
    for i, lf in enumerate(leaves):
        s, e = lf["range"]
        Q[s:e] = thin_q(lf["V"], lf["tau"]) @ Qtree[i * d:(i + 1) * d].astype(leaf_dtype)
    Q, R = normalise(Q, root["R"])
    return {"R": R, "Q": Q, "leaves": leaves, "levels": levels}
