"""FP64 / exact oracle of the tuning objective (test infrastructure only).

Section 5.2 tunes the threshold and the gap penalty by drawing parameter
values at random and keeping those whose automatic alignment of sample
article pairs is most similar to a human alignment of them; the similarity is
a percentage, and the comparison of the two alignments is made with a
Needleman-Wunsch alignment.

Reading (the paper gives no formula): an alignment is the sequence of its
links (i, j) in path order; the two sequences are aligned by Needleman-Wunsch
with score 1 for identical links, 0 otherwise and no gap cost (a longest
common subsequence), and the similarity is 2 * matched / (|auto| + |human|)
(the Dice coefficient, which equals the micro-F1 of the links).  For two
monotone link lists (both strictly increasing in i and in j, as every
Needleman-Wunsch path is) the matched count is the size of their
intersection; the tests pin that reduction, which the GPU evaluation uses.
"""
from __future__ import annotations


def nw_matched(auto, human) -> int:
    """Needleman-Wunsch (LCS) alignment of two link sequences: the number of
    identical links it pairs up.  Plain O(|auto| * |human|) table."""
    a = [tuple(x) for x in auto]
    h = [tuple(x) for x in human]
    prev = [0] * (len(h) + 1)
    for x in a:
        cur = [0] * (len(h) + 1)
        for k, y in enumerate(h, start=1):
            cur[k] = max(prev[k], cur[k - 1], prev[k - 1] + (1 if x == y else 0))
        prev = cur
    return prev[-1]


def similarity(auto_pairs, human_pairs) -> dict:
    """Micro-averaged similarity of automatic and human alignments over a set
    of document pairs: matched links (NW alignment per pair), links of each
    side, and the percentage 2 * matched / (|auto| + |human|)."""
    m = na = nh = 0
    for auto, human in zip(auto_pairs, human_pairs):
        m += nw_matched(auto, human)
        na += len(auto)
        nh += len(human)
    return {"matched": m, "auto": na, "human": nh, "similarity": 2.0 * m / (na + nh) if na + nh else 0.0}
