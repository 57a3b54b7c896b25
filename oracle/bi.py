"""Oracle of bi-directional mining (test infrastructure only).

Section 5.4 mines with a second classifier trained for the reverse language
direction ("BI", next to the one-directional "MONO") and keeps the
bi-sentences of both, repetitions removed.  Reading: the reverse direction is
the same method with the two corpora swapped and a dictionary from target ids
to source ids, under its own parameters; the links of a pair from the two
directions (the reverse ones mapped back to forward coordinates) are combined
as a union (BI) or, for a stricter filter, an intersection, ordered by (i, j).
Plain Python over the definitions; the reverse mining itself is ``oracle.mine``
on the reversed batch.
"""
from __future__ import annotations

import math

import numpy as np

from paper_1512_01641_gb300 import synth


def transpose_dictionary(dic: synth.Dictionary) -> synth.Dictionary:
    """For every target id t, the ascending source ids v with t among v's
    translations."""
    lists = [[] for _ in range(dic.v_tgt)]
    for v in range(dic.v_src):
        for t in dic.tgt[dic.off[v]:dic.off[v + 1]]:
            lists[int(t)].append(v)
    off = np.zeros(dic.v_tgt + 1, np.int32)
    off[1:] = np.cumsum([len(x) for x in lists])
    tgt = np.array([v for x in lists for v in x], np.int32)
    return synth.Dictionary(dic.v_tgt, dic.v_src, off, tgt)


def reversed_batch(batch: synth.Batch, dic_rev: synth.Dictionary | None = None) -> synth.Batch:
    """The same pairs with the roles swapped: target documents become the
    source; the dictionary maps target ids to source ids."""
    d = dic_rev if dic_rev is not None else transpose_dictionary(batch.dic)
    gold = [np.ascontiguousarray(g[:, ::-1]) for g in batch.gold] if batch.gold else []
    return synth.Batch(batch.tgt, batch.src, d, batch.planted, gold)


def combine(links_fwd, links_rev, mode: str = "union"):
    """Per pair: the forward links (i, j, s) and the reverse links (i', j', s')
    -> the union (or intersection) of the links (i, j) = forward or (j', i')
    = reverse, ascending in (i, j), as (i, j, s_fwd, s_rev) with NaN where a
    direction did not keep the link."""
    out = []
    for fw, rv in zip(links_fwd, links_rev):
        f = {(int(i), int(j)): s for i, j, s in fw}
        r = {(int(j), int(i)): s for i, j, s in rv}
        keys = (set(f) | set(r)) if mode == "union" else (set(f) & set(r))
        out.append([(i, j, f.get((i, j), math.nan), r.get((i, j), math.nan)) for i, j in sorted(keys)])
    return out
