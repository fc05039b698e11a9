"""Node geometry helpers shared by the tests (no arithmetic of the method)."""
import numpy as np


def coincident_pairs(lxy):
    """((leaf_a, leaf_b), (node_a, node_b)) index arrays of the nodes that two
    leaves share: the corner-free edge nodes of every interior leaf edge.
    lxy is [leaves][nodes][2]; coordinates are matched after rounding to 12
    decimals, and no point may belong to more than two leaves."""
    leaves, n, _ = lxy.shape
    key = np.round(lxy.reshape(-1, 2), 12)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    inv = inv.ravel()
    order = np.argsort(inv, kind="stable")
    groups = np.split(order, np.cumsum(cnt)[:-1])
    assert all(len(g) <= 2 for g in groups)
    pairs = np.array([g for g in groups if len(g) == 2]).reshape(-1, 2)
    return (pairs // n).T, (pairs % n).T
