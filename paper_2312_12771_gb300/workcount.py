"""Algorithmic work of the band factorisation (host logic, no method arithmetic).

The factor's algorithmic flop count is that of the sparse Cholesky of K_mm in
the folded periodic ordering: with c_j the number of nonzeros of column j of L
below the diagonal, sum_j (c_j^2 + 2 c_j + 1) for the factorisation and
sum_j (2 c_j + 1) per right-hand side for each triangular solve.  The band
kernels compute every entry of the band (half width kd = 4N + 5 in 2D); the
column counts here come from a symbolic factorisation of the sparsity pattern
(elimination tree, children's row sets merged into their parent), so entries
of the band that stay zero are not counted as work.
"""
from __future__ import annotations

import functools

import numpy as np


def fold_pos(i: int, N: int) -> int:
    """Folded position of grid index i: 0, 1, N-1, 2, N-2, ... get 0, 1, 2, 3, 4, ..."""
    if i == 0:
        return 0
    return 2 * i - 1 if 2 * i <= N else 2 * (N - i)


def kmm_lower_pattern(N: int, d: int) -> list[list[int]]:
    """For each reduced DOF j (folded node order, corner node pinned, DOF d(q-1)+c),
    the rows i > j coupled to it in K_mm (nodes of the 3^d periodic neighbourhood)."""
    nn = N ** d
    unfold = [0] * N
    for i in range(N):
        unfold[fold_pos(i, N)] = i
    nm = d * (nn - 1)
    rows = [set() for _ in range(nm)]
    for q in range(1, nn):
        g = [unfold[(q // N ** k) % N] for k in range(d)]
        for off in range(3 ** d):
            h = [(g[k] + (off // 3 ** k) % 3 - 1) % N for k in range(d)]
            qn = sum(fold_pos(h[k], N) * N ** k for k in range(d))
            if qn == 0:
                continue
            for c in range(d):
                for c2 in range(d):
                    j, i = d * (q - 1) + c, d * (qn - 1) + c2
                    if i > j:
                        rows[j].add(i)
    return [sorted(r) for r in rows]


def column_structures(N: int, d: int = 2) -> list[np.ndarray]:
    """Rows below the diagonal of each column of the Cholesky factor of K_mm (the
    symbolic factorisation: own pattern plus the row sets of the eliminated children)."""
    low = kmm_lower_pattern(N, d)
    n = len(low)
    pending: dict[int, set] = {}   # column -> rows contributed by its eliminated children
    out = []
    for j in range(n):
        s = set(low[j])
        s |= pending.pop(j, set())
        s.discard(j)
        out.append(np.array(sorted(s), dtype=np.int64))
        if s:
            parent = min(s)
            s.discard(parent)
            pending.setdefault(parent, set()).update(s)
    return out


@functools.lru_cache(maxsize=None)
def column_counts(N: int, d: int = 2) -> np.ndarray:
    """Nonzeros below the diagonal in each column of the Cholesky factor of K_mm."""
    return np.array([len(c) for c in column_structures(N, d)], dtype=np.int64)


def factor_flops(N: int, d: int = 2, nr: int | None = None) -> tuple[float, float]:
    """(flops of the factorisation with the forward elimination of nr right-hand
    sides, flops of one triangular solve with one right-hand side)."""
    if nr is None:
        nr = d * d + 1
    c = column_counts(N, d).astype(np.float64)
    chol = float(np.sum(c * c + 2 * c + 1))
    tri = float(np.sum(2 * c + 1))
    return chol + nr * tri, tri
