"""Brute-force enumeration of every monotone alignment (test infrastructure).

An alignment of N source and M target sentences is a path from (0,0) to (N,M)
with unit steps DIAG (1,1), UP (1,0) and LEFT (0,1) -- the paths that
Needleman-Wunsch ranges over (Section 5.1; no crossings and no going back,
which is the constraint the paper contrasts with unconstrained A*).  There are
Delannoy(N, M) of them.  Its score is the sum of the similarities of its DIAG
cells minus the gap penalty for every UP or LEFT step.

Pure Python loops: for N, M <= 8 only.
"""
from __future__ import annotations

import math
from functools import lru_cache


@lru_cache(maxsize=None)
def delannoy(m: int, n: int) -> int:
    """Number of monotone lattice paths with unit E, N and NE steps."""
    return sum(math.comb(m, k) * math.comb(n, k) * 2 ** k for k in range(min(m, n) + 1))


def alignments(N: int, M: int):
    """Yield every alignment as a tuple of 0-based DIAG cells (ascending), and
    the number of gap steps it takes."""
    stack = [(0, 0, ())]
    while stack:
        i, j, diag = stack.pop()
        if i == N and j == M:
            yield diag, N + M - 2 * len(diag)
            continue
        if i < N and j < M:
            stack.append((i + 1, j + 1, diag + ((i, j),)))
        if i < N:
            stack.append((i + 1, j, diag))
        if j < M:
            stack.append((i, j + 1, diag))


def score(s, p, diag, n_gaps) -> float:
    return sum(s[i][j] for (i, j) in diag) - p * n_gaps


def hard(s, p):
    """(best score, list of optimal DIAG sets) over all alignments."""
    N, M = len(s), len(s[0]) if len(s) else 0
    best, arg = -math.inf, []
    for diag, g in alignments(N, M):
        v = score(s, p, diag, g)
        if v > best:
            best, arg = v, [diag]
        elif v == best:
            arg.append(diag)
    return best, arg


def soft(s, p, gamma):
    """(gamma * log sum_paths exp(score/gamma), marginals E[i][j]) by enumeration.
    E[i][j] is the probability, under the Gibbs distribution over paths, that
    the path takes cell (i, j) diagonally; it equals dV/ds_ij."""
    N, M = len(s), len(s[0]) if len(s) else 0
    scores = [(score(s, p, d, g), d) for d, g in alignments(N, M)]
    mx = max(v for v, _ in scores)
    Z = 0.0
    E = [[0.0] * M for _ in range(N)]
    for v, d in scores:
        w = math.exp((v - mx) / gamma)
        Z += w
        for (i, j) in d:
            E[i][j] += w
    for i in range(N):
        for j in range(M):
            E[i][j] /= Z
    return mx + gamma * math.log(Z), E


def unconstrained_choices(N: int, M: int):
    """Every row-by-row choice of the unconstrained aligner's move set: each
    source row unmatched (None) or matched to any target column, in any
    order -- (M + 1) ** N of them."""
    import itertools
    return itertools.product([None] + list(range(M)), repeat=N)
