"""FP64 reference of the unconstrained (Yalign A*) sentence aligner (test
infrastructure only).

Section 4 says Yalign aligned sentences with an A* search that maximises the
sum of pair similarities; Section 5.1 says that with Needleman-Wunsch's
similarities and gap penalty A* gives NW's result only if its paths may not
go up or left in the S matrix, that Yalign imposes no such constraint, and
that every move up or left comes back into a sequence, so that a phrase can
be used twice (Figures 3 and 5 against Figures 4 and 6).  The paper gives no
cost model for those moves.  Reading used here (it reproduces Figure 3's path
and alignment exactly):

  * source sentences (rows) are taken in order; each is either left
    unmatched (-p, the target pointer stays) or matched to a target
    sentence (column) c';
  * a match ahead of the pointer c (c' > c) is the NW diagonal step after
    c' - c - 1 unmatched target sentences (-p each);
  * a match at or behind the pointer (c' <= c) goes back into the target
    sequence: s(i, c') - p, one gap penalty for the move back;
  * target sentences after the final pointer are unmatched (-p each).

Forbidding the move back leaves exactly the NW alignments and their scores.
Exact ties in the traceback prefer, as NW's rule does, the gap: unmatched
before a forward match before a move back; among forward matches the nearest
predecessor pointer, among moves back the nearest; at the end the smallest
final pointer.

Plain Python loops in definition order: O(N M^2), for small pairs only.
"""
from __future__ import annotations

import math

import numpy as np

NEG = -math.inf


def fill(s, p, back=True):
    """Best scores A[i][c] (rows 0..N processed, target pointer c in 0..M) and
    the predecessor pointer of each state (-1: row i left unmatched).  With
    back=False the move back is not offered (the Needleman-Wunsch paths)."""
    s = np.asarray(s, np.float64)
    N, M = s.shape
    A = [[NEG] * (M + 1) for _ in range(N + 1)]
    prev = [[-2] * (M + 1) for _ in range(N + 1)]
    A[0][0] = 0.0
    for i in range(1, N + 1):
        for c2 in range(M + 1):
            best, arg = NEG, -2
            if A[i - 1][c2] > NEG:  # row i unmatched, pointer stays
                best, arg = A[i - 1][c2] - p, -1
            if c2 >= 1:
                sim = s[i - 1][c2 - 1]
                for c in range(c2 - 1, -1, -1):  # forward match, nearest pointer first
                    if A[i - 1][c] > NEG:
                        v = A[i - 1][c] + sim - p * (c2 - c - 1)
                        if v > best:
                            best, arg = v, c
                for c in range(c2, M + 1 if back else c2):  # move back, nearest pointer first
                    if A[i - 1][c] > NEG:
                        v = A[i - 1][c] + sim - p
                        if v > best:
                            best, arg = v, c
            A[i][c2] = best
            prev[i][c2] = arg
    return A, prev


def align(s, p, back=True):
    """(score, links): links are the matched (row, column) cells, 0-based, in
    row order (columns need not increase)."""
    s = np.asarray(s, np.float64)
    N, M = s.shape
    A, prev = fill(s, p, back)
    c_end, best = 0, NEG
    for c in range(M + 1):
        v = A[N][c] - p * (M - c)
        if v > best:
            best, c_end = v, c
    links = []
    c = c_end
    for i in range(N, 0, -1):
        a = prev[i][c]
        if a != -1:
            links.append((i - 1, c - 1))
            c = a
    links.reverse()
    return best, links


def path_score(s, p, choice) -> float:
    """Score of one row-by-row choice (choice[i] = matched column, 0-based, or
    None) under the cost model above."""
    s = np.asarray(s, np.float64)
    N, M = s.shape
    c, tot = 0, 0.0
    for i, j in enumerate(choice):
        if j is None:
            tot -= p
            continue
        c2 = j + 1
        tot += s[i, j] - (p * (c2 - c - 1) if c2 > c else p)
        c = c2
    return tot - p * (M - c)
