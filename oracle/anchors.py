"""Oracle of the anchor tokens of Section 5.3 (test infrastructure only).

Section 5.3 observes that names, dates, numbers and references that two
Wikipedia sentences share mark them as likely translations, and that they
should be analysed beside the other comparison techniques.  Reading: such an
anchor is the same token in both languages, so it takes part in the overlap
counts of Section 4 as a word whose translation is itself.  Anchor a of a
source sentence becomes source token v_src + a, of a target sentence target
token v_tgt + a, and the dictionary gains the entries v_src + a -> {v_tgt + a}.
Plain Python over the definitions (sorted token lists, CSR arrays).
"""
from __future__ import annotations

import numpy as np

from paper_1512_01641_gb300 import synth


def _extend_corpus(c: synth.Corpus, anc: synth.Anchors, v_words: int) -> synth.Corpus:
    n = len(c.sent_tok_off) - 1
    lens, toks = [], []
    for s in range(n):
        words = c.tok[c.sent_tok_off[s]:c.sent_tok_off[s + 1]].tolist()
        extra = [v_words + int(a) for a in anc.ids[anc.sent_off[s]:anc.sent_off[s + 1]]]
        t = sorted(words + extra)
        lens.append(len(t))
        toks.extend(t)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(lens)
    return synth.Corpus(c.doc_sent_off.copy(), off, np.asarray(toks, np.int32))


def extend_dictionary(dic: synth.Dictionary, v_anchor: int) -> synth.Dictionary:
    lists = [dic.tgt[dic.off[v]:dic.off[v + 1]].tolist() for v in range(dic.v_src)]
    lists += [[dic.v_tgt + a] for a in range(v_anchor)]
    off = np.zeros(len(lists) + 1, np.int32)
    off[1:] = np.cumsum([len(x) for x in lists])
    return synth.Dictionary(dic.v_src + v_anchor, dic.v_tgt + v_anchor, off,
                            np.asarray([t for x in lists for t in x], np.int32))


def extend_batch(batch: synth.Batch, src_anchors: synth.Anchors, tgt_anchors: synth.Anchors,
                 v_anchor: int) -> synth.Batch:
    """The batch with every sentence's anchors among its tokens and the
    identity entries of the anchors in the dictionary."""
    return synth.Batch(_extend_corpus(batch.src, src_anchors, batch.dic.v_src),
                       _extend_corpus(batch.tgt, tgt_anchors, batch.dic.v_tgt),
                       extend_dictionary(batch.dic, v_anchor), batch.planted, batch.gold)


def shared_positions(a_src, a_tgt) -> tuple[int, int]:
    """(source anchor positions whose anchor the target sentence carries,
    target anchor positions whose anchor the source sentence carries)."""
    s, t = set(int(x) for x in a_src), set(int(x) for x in a_tgt)
    return sum(1 for x in a_src if int(x) in t), sum(1 for x in a_tgt if int(x) in s)
