"""Determinism check of the GPU inner product (not an oracle): the library reduces every inner
product in one fixed order -- leaves of 16 consecutive products summed left to right, the leaf
sums combined by a stride-doubling pairwise tree (level d adds s_{j+d} into s_j for j a multiple
of 2d with j + d < m) -- so its result depends on n only.  This restates that order with the
oracle's scalar operations, to check the kernel's bits; the oracle's own inner product is the
plain left-to-right sum.
"""
import numpy as np

import oracle

LEAF = 16


def tree_dot(a, b, n, w, c=1):
    s = c * w
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m = (n + LEAF - 1) // LEAF
    if n <= 0:
        return np.zeros(s)
    # a leaf summed left to right from 0 equals the leaf summed from its first product (0 + p = p
    # exactly in every format)
    leaf = [oracle.dot(a[j * LEAF * s:min(n, (j + 1) * LEAF) * s], b[j * LEAF * s:min(n, (j + 1) * LEAF) * s],
                       min(n, (j + 1) * LEAF) - j * LEAF, w, c) for j in range(m)]
    d = 1
    while d < m:
        for j in range(0, m - d, 2 * d):
            x, y = leaf[j], leaf[j + d]
            leaf[j] = np.concatenate([oracle.mp_op("add", w, x[p * w:(p + 1) * w], y[p * w:(p + 1) * w])
                                      for p in range(c)])
        d *= 2
    return leaf[0]
