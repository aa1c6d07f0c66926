"""Helpers shared by the GPU tests: device copies and error measures."""
import numpy as np

import oracle as O

U2 = 2.0 ** -106  # u^2 for binary64
Q2 = 2.0 ** -212


def to_dev(M):
    import torch
    return torch.from_numpy(np.ascontiguousarray(M)).cuda()


def to_host(T):
    return T.cpu().numpy()


def absprod(A, B, rows=None, cols=None):
    """sum_k |a_ik| |b_kj| in double from the leading limbs (elementwise scale)."""
    a, b = np.abs(A[0]), np.abs(B[0])
    if rows is None:
        return a @ b
    return np.einsum("tk,kt->t", a[rows], b[:, cols])


def sample_entries(m, n, count, seed):
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, m, size=count)
    cols = rng.integers(0, n, size=count)
    # always include the corners and the last row / column (ragged tails)
    rows = np.concatenate([rows, [0, m - 1, m - 1, 0]])
    cols = np.concatenate([cols, [0, n - 1, 0, n - 1]])
    return rows.astype(np.int64), cols.astype(np.int64)


def normwise_bound(l, limbs, algo):
    eps = 2.0 ** -104 if limbs == 2 else 2.0 ** -208
    if algo in ("strassen", "winograd"):
        return 8 * l ** np.log2(12) * eps
    return 8 * l * eps
