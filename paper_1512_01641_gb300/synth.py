"""Seeded synthetic comparable corpora shaped like topic-aligned Wikipedia article pairs.

This module only draws random inputs; it holds none of the mining arithmetic
(no overlap counting, no scoring, no alignment).  Both the CUDA path and the
FP64 oracle are fed from it.

The paper mines topic-aligned Wikipedia article pairs (Section 4) with a
bilingual 1-gram dictionary taken from a phrase table (Section 4).  Neither the
articles nor the dictionary are available, so these stand in for them:

* a sentence is a list of 5..30 token ids (uniform length), drawn Zipf(s) over
  a per-language vocabulary and stored sorted ascending;
* the dictionary maps each source id to 1..3 distinct, uniformly drawn target
  ids (sorted);
* document sizes are lognormal (median 60 sentences, sigma 0.8, clipped to
  5..800), source and target sized independently for unrelated pairs;
* a "planted" pair builds its target document from the source document:
  each source sentence is dropped with probability ``p_sdrop``; each token of
  a kept sentence is dropped with probability ``p_wdrop`` and otherwise mapped
  to one uniformly chosen translation; the result is re-sorted (a sentence
  left empty keeps one translated token of a random source position);
  ``round(p_ins * N)`` random sentences are inserted at uniformly chosen
  positions.  Gold links are (source sentence, target position of its
  translation); they are monotone by construction.

All draws come from one NumPy PCG64 stream per call, so a (config, seed) pair
fixes every byte.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

MIN_LEN, MAX_LEN = 5, 30


@dataclass
class Corpus:
    """CSR corpus: document d owns sentences doc_sent_off[d]:doc_sent_off[d+1];
    sentence s owns tokens tok[sent_tok_off[s]:sent_tok_off[s+1]] (sorted)."""
    doc_sent_off: np.ndarray  # int64, n_docs+1
    sent_tok_off: np.ndarray  # int64, n_sents+1
    tok: np.ndarray           # int32

    @property
    def n_docs(self) -> int:
        return len(self.doc_sent_off) - 1

    def doc_sizes(self) -> np.ndarray:
        return np.diff(self.doc_sent_off)

    def sentence(self, s: int) -> np.ndarray:
        return self.tok[self.sent_tok_off[s]:self.sent_tok_off[s + 1]]

    def doc(self, d: int) -> list:
        a, b = self.doc_sent_off[d], self.doc_sent_off[d + 1]
        return [self.sentence(s) for s in range(a, b)]

    def subset(self, docs) -> "Corpus":
        """A new corpus holding only the listed documents, in that order."""
        docs = np.asarray(docs, dtype=np.int64)
        sizes = self.doc_sizes()[docs]
        doc_off = np.zeros(len(docs) + 1, np.int64)
        np.cumsum(sizes, out=doc_off[1:])
        sents = np.concatenate([np.arange(self.doc_sent_off[d], self.doc_sent_off[d + 1])
                                for d in docs]) if len(docs) else np.zeros(0, np.int64)
        lens = (self.sent_tok_off[sents + 1] - self.sent_tok_off[sents]) if len(sents) else np.zeros(0, np.int64)
        tok_off = np.zeros(len(sents) + 1, np.int64)
        np.cumsum(lens, out=tok_off[1:])
        if len(sents):
            starts = self.sent_tok_off[sents]
            idx = np.repeat(starts - tok_off[:-1], lens) + np.arange(tok_off[-1])
            tok = self.tok[idx]
        else:
            tok = np.zeros(0, np.int32)
        return Corpus(doc_off, tok_off, tok.astype(np.int32))


@dataclass
class Dictionary:
    """CSR bilingual dictionary: source id v maps to tgt[off[v]:off[v+1]]
    (sorted, distinct target ids)."""
    v_src: int
    v_tgt: int
    off: np.ndarray  # int32, v_src+1
    tgt: np.ndarray  # int32

    def translations(self, v: int) -> np.ndarray:
        return self.tgt[self.off[v]:self.off[v + 1]]


@dataclass
class Batch:
    src: Corpus
    tgt: Corpus
    dic: Dictionary
    planted: np.ndarray                     # bool per pair
    gold: list = field(default_factory=list)  # per pair: int32 array (k,2) of (i,j), empty if unplanted

    @property
    def n_pairs(self) -> int:
        return self.src.n_docs

    def cells(self) -> int:
        return int((self.src.doc_sizes() * self.tgt.doc_sizes()).sum())

    def subset(self, pairs) -> "Batch":
        pairs = np.asarray(pairs, dtype=np.int64)
        return Batch(self.src.subset(pairs), self.tgt.subset(pairs), self.dic,
                     self.planted[pairs], [self.gold[k] for k in pairs] if self.gold else [])


# --------------------------------------------------------------------------
# samplers
# --------------------------------------------------------------------------
class ZipfAlias:
    """Walker/Vose alias table for P(id = r-1) proportional to r^-s, r = 1..v."""

    def __init__(self, v: int, s: float):
        p = np.arange(1, v + 1, dtype=np.float64) ** (-s)
        p /= p.sum()
        n = v
        prob = p * n
        alias = np.zeros(n, np.int64)
        small = [i for i in range(n) if prob[i] < 1.0]
        large = [i for i in range(n) if prob[i] >= 1.0]
        prob = prob.tolist()
        while small and large:
            l = small.pop()
            g = large.pop()
            alias[l] = g
            prob[g] = prob[g] + prob[l] - 1.0
            (small if prob[g] < 1.0 else large).append(g)
        for i in large + small:
            prob[i] = 1.0
        self.v = v
        self.prob = np.asarray(prob)
        self.alias = alias

    def draw(self, rng: np.random.Generator, n: int) -> np.ndarray:
        col = rng.integers(0, self.v, size=n)
        u = rng.random(n)
        return np.where(u < self.prob[col], col, self.alias[col]).astype(np.int32)


def make_dictionary(rng: np.random.Generator, v_src: int, v_tgt: int,
                    kmin: int = 1, kmax: int = 3) -> Dictionary:
    """Each source id gets U{kmin..kmax} distinct uniform target ids, sorted."""
    k = rng.integers(kmin, kmax + 1, size=v_src)
    off = np.zeros(v_src + 1, np.int64)
    np.cumsum(k, out=off[1:])
    total = int(off[-1])
    tgt = rng.integers(0, v_tgt, size=total).astype(np.int64)
    # resample duplicates inside a list until all lists are distinct
    owner = np.repeat(np.arange(v_src), k)
    while True:
        key = owner * v_tgt + tgt
        order = np.lexsort((tgt, owner))
        ks = key[order]
        dup = np.zeros(total, bool)
        dup[order[1:][ks[1:] == ks[:-1]]] = True
        nd = int(dup.sum())
        if nd == 0:
            break
        tgt[dup] = rng.integers(0, v_tgt, size=nd)
    order = np.lexsort((tgt, owner))
    tgt = tgt[order]
    return Dictionary(v_src, v_tgt, off.astype(np.int32), tgt.astype(np.int32))


def thin_dictionary(dic: Dictionary, p_drop: float, seed: int) -> Dictionary:
    """A copy of the dictionary with each entry dropped with probability
    p_drop (lists may become empty): the incomplete dictionary a miner works
    with when the data were made with the full one."""
    rng = np.random.Generator(np.random.PCG64(seed))
    keep = rng.random(len(dic.tgt)) >= p_drop
    owner = np.repeat(np.arange(dic.v_src), np.diff(dic.off.astype(np.int64)))
    off = np.zeros(dic.v_src + 1, np.int64)
    np.cumsum(np.bincount(owner[keep], minlength=dic.v_src), out=off[1:])
    return Dictionary(dic.v_src, dic.v_tgt, off.astype(np.int32), dic.tgt[keep].astype(np.int32))


def lognormal_sizes(rng: np.random.Generator, n: int, median: float = 60.0,
                    sigma: float = 0.8, lo: int = 5, hi: int = 800) -> np.ndarray:
    x = rng.lognormal(mean=np.log(median), sigma=sigma, size=n)
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def _sort_segments(tok: np.ndarray, lens: np.ndarray) -> np.ndarray:
    """Sort each sentence's tokens ascending (sentences are at most MAX_LEN long)."""
    n = len(lens)
    if n == 0:
        return tok
    width = int(lens.max())
    pad = np.full((n, width), np.iinfo(np.int32).max, np.int32)
    off = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    col = np.arange(len(tok)) - np.repeat(off[:-1], lens)
    row = np.repeat(np.arange(n), lens)
    pad[row, col] = tok
    pad.sort(axis=1)
    return pad[row, col]


def _random_sentences(rng, zipf: ZipfAlias, n_sent: int):
    lens = rng.integers(MIN_LEN, MAX_LEN + 1, size=n_sent).astype(np.int64)
    tok = zipf.draw(rng, int(lens.sum()))
    return lens, tok


def _csr(lens: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    return off


# --------------------------------------------------------------------------
# batch builder
# --------------------------------------------------------------------------
def make_batch(seed: int, n_pairs: int, *, v_src: int = 50_000, v_tgt: int = 50_000,
               zipf_s: float = 1.1, planted_frac: float = 0.5,
               p_wdrop: float = 0.2, p_sdrop: float = 0.2, p_ins: float = 0.2,
               src_sizes=None, tgt_sizes=None, dic: Dictionary | None = None,
               size_median: float = 60.0, size_sigma: float = 0.8,
               size_lo: int = 5, size_hi: int = 800,
               keep_square: np.ndarray | None = None) -> Batch:
    """Build ``n_pairs`` document pairs.

    src_sizes / tgt_sizes: explicit sentence counts (default lognormal).  For a
    planted pair the target size follows from dropping and inserting, unless
    ``keep_square[k]`` is set, in which case the number of inserted sentences
    is chosen so that the target has as many sentences as the source.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if dic is None:
        dic = make_dictionary(rng, v_src, v_tgt)
    zs = ZipfAlias(dic.v_src, zipf_s)
    zt = ZipfAlias(dic.v_tgt, zipf_s)

    if src_sizes is None:
        N = lognormal_sizes(rng, n_pairs, size_median, size_sigma, size_lo, size_hi)
    else:
        N = np.asarray(src_sizes, np.int64)
    n_plant = int(round(planted_frac * n_pairs))
    planted = np.zeros(n_pairs, bool)
    planted[rng.permutation(n_pairs)[:n_plant]] = True
    if keep_square is None:
        keep_square = np.zeros(n_pairs, bool)

    # ---- source corpus
    s_lens, s_tok = _random_sentences(rng, zs, int(N.sum()))
    s_tok = _sort_segments(s_tok, s_lens)
    src = Corpus(_csr(N), _csr(s_lens), s_tok)

    # ---- target documents: sizes and slot contents
    pair_of_src = np.repeat(np.arange(n_pairs), N)
    keep = (rng.random(int(N.sum())) >= p_sdrop) & planted[pair_of_src]
    K = np.bincount(pair_of_src, weights=keep, minlength=n_pairs).astype(np.int64)
    if tgt_sizes is None:
        M_rand = lognormal_sizes(rng, n_pairs, size_median, size_sigma, size_lo, size_hi)
    else:
        M_rand = np.asarray(tgt_sizes, np.int64)
    n_ins = np.where(keep_square, np.maximum(N - K, 0), np.rint(p_ins * N).astype(np.int64))
    M = np.where(planted, K + n_ins, M_rand)
    if np.any(M == 0):  # a planted document that lost everything gets one noise sentence
        n_ins = np.where(planted & (M == 0), 1, n_ins)
        M = np.where(planted, K + n_ins, M_rand)

    # per target slot: source sentence index (global) or -1 for a random sentence
    n_tslots = int(M.sum())
    slot_pair = np.repeat(np.arange(n_pairs), M)
    slot_src = np.full(n_tslots, -1, np.int64)
    tdoc_off = _csr(M)
    if n_plant:
        # choose which slots of a planted doc are inserted: the n_ins smallest random keys
        key = rng.random(n_tslots)
        order = np.lexsort((key, slot_pair))
        rank = np.empty(n_tslots, np.int64)
        rank[order] = np.arange(n_tslots) - np.repeat(tdoc_off[:-1], M)
        is_ins = planted[slot_pair] & (rank < n_ins[slot_pair])
        trans_slot = planted[slot_pair] & ~is_ins
        # kept src sentences fill the translated slots in order
        kept_src = np.nonzero(keep)[0]
        slot_src[np.nonzero(trans_slot)[0]] = kept_src
    # ---- target sentence tokens
    t_lens = np.zeros(n_tslots, np.int64)
    rand_slots = np.nonzero(slot_src < 0)[0]
    r_lens, r_tok = _random_sentences(rng, zt, len(rand_slots))
    t_lens[rand_slots] = r_lens
    tr_slots = np.nonzero(slot_src >= 0)[0]
    tr_tok_list = np.zeros(0, np.int32)
    if len(tr_slots):
        srcs = slot_src[tr_slots]
        sl = s_lens[srcs]
        tok_idx = np.repeat(src.sent_tok_off[srcs], sl) + (np.arange(int(sl.sum())) - np.repeat(_csr(sl)[:-1], sl))
        stoks = s_tok[tok_idx]
        kept_tok = rng.random(len(stoks)) >= p_wdrop
        cnt = (dic.off[stoks + 1] - dic.off[stoks]).astype(np.int64)
        pick = (rng.random(len(stoks)) * cnt).astype(np.int64)
        trans = dic.tgt[dic.off[stoks] + pick]
        sent_of_tok = np.repeat(np.arange(len(tr_slots)), sl)
        n_kept = np.bincount(sent_of_tok, weights=kept_tok, minlength=len(tr_slots)).astype(np.int64)
        empty = np.nonzero(n_kept == 0)[0]
        if len(empty):  # keep one translated token of a random position
            pos = (rng.random(len(empty)) * sl[empty]).astype(np.int64)
            kept_tok[_csr(sl)[:-1][empty] + pos] = True
            n_kept[empty] = 1
        t_lens[tr_slots] = n_kept
        tr_tok_list = trans[kept_tok].astype(np.int32)
    # assemble target tokens in slot order
    t_off = _csr(t_lens)
    t_tok = np.zeros(int(t_off[-1]), np.int32)
    if len(rand_slots):
        idx = np.repeat(t_off[rand_slots], r_lens) + (np.arange(int(r_lens.sum())) - np.repeat(_csr(r_lens)[:-1], r_lens))
        t_tok[idx] = r_tok
    if len(tr_slots):
        tl = t_lens[tr_slots]
        idx = np.repeat(t_off[tr_slots], tl) + (np.arange(int(tl.sum())) - np.repeat(_csr(tl)[:-1], tl))
        t_tok[idx] = tr_tok_list
    t_tok = _sort_segments(t_tok, t_lens)
    tgt = Corpus(tdoc_off, t_off, t_tok)

    # ---- gold links (per planted pair, local indices)
    gold = []
    src_local = np.arange(int(N.sum())) - np.repeat(src.doc_sent_off[:-1], N)
    tr_local = tr_slots - tdoc_off[slot_pair[tr_slots]] if len(tr_slots) else tr_slots
    gsrc = src_local[slot_src[tr_slots]] if len(tr_slots) else tr_slots
    gpair = slot_pair[tr_slots] if len(tr_slots) else tr_slots
    goff = _csr(np.bincount(gpair, minlength=n_pairs)) if len(tr_slots) else np.zeros(n_pairs + 1, np.int64)
    for k in range(n_pairs):
        a, b = goff[k], goff[k + 1]
        gold.append(np.stack([gsrc[a:b], tr_local[a:b]], axis=1).astype(np.int32) if b > a
                    else np.zeros((0, 2), np.int32))
    return Batch(src, tgt, dic, planted, gold)


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------
SEED_BASE = 20151205


def single_pair(seed: int = SEED_BASE + 0) -> Batch:
    """One unplanted pair, 40 x 45 sentences, 20k-id vocabularies."""
    return make_batch(seed, 1, v_src=20_000, v_tgt=20_000, planted_frac=0.0,
                      src_sizes=[40], tgt_sizes=[45])


def wiki_batch(n_pairs: int = 10_000, seed: int = SEED_BASE + 1) -> Batch:
    """n_pairs Wikipedia-shaped pairs (lognormal sizes), half planted, 50k vocab."""
    return make_batch(seed, n_pairs)


def uneven_batch(n_pairs: int = 100_000, n_long: int = 8, long_n: int = 5000,
                 seed: int = SEED_BASE + 2) -> Batch:
    """n_pairs Wikipedia-shaped pairs followed by n_long pairs of long_n x long_n
    sentences (every other long pair planted, target kept square)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1_000_003))
    dic = make_dictionary(rng, 50_000, 50_000)
    a = make_batch(seed, n_pairs, dic=dic) if n_pairs else None
    if n_long == 0:
        return a
    sz = np.full(n_long, long_n)
    b = make_batch(seed + 7, n_long, dic=dic, src_sizes=sz, tgt_sizes=sz,
                   keep_square=np.ones(n_long, bool))
    return b if a is None else concat_batches(a, b)


def soft_batch(n_pairs: int = 4096, n: int = 100, seed: int = SEED_BASE + 3) -> Batch:
    """Planted pairs of n source sentences (about n x n after drops/inserts)."""
    return make_batch(seed, n_pairs, planted_frac=1.0, src_sizes=np.full(n_pairs, n))


def tune_batch(n_pairs: int = 50_000, seed: int = SEED_BASE + 4, dic=None) -> Batch:
    """Planted pairs, lognormal sizes, 30% inserted noise sentences, 25% word dropout."""
    return make_batch(seed, n_pairs, planted_frac=1.0, p_ins=0.3, p_wdrop=0.25, dic=dic)


def concat_corpora(a: Corpus, b: Corpus) -> Corpus:
    doc = np.concatenate([a.doc_sent_off, b.doc_sent_off[1:] + a.doc_sent_off[-1]])
    sent = np.concatenate([a.sent_tok_off, b.sent_tok_off[1:] + a.sent_tok_off[-1]])
    return Corpus(doc, sent, np.concatenate([a.tok, b.tok]))


def concat_batches(a: Batch, b: Batch) -> Batch:
    assert a.dic is b.dic
    return Batch(concat_corpora(a.src, b.src), concat_corpora(a.tgt, b.tgt), a.dic,
                 np.concatenate([a.planted, b.planted]), a.gold + b.gold)


def from_lists(src_docs, tgt_docs, dic_lists, v_tgt=None) -> Batch:
    """Build a batch from Python lists (tests): src_docs[k] = list of token lists."""
    def corpus(docs):
        sizes = [len(d) for d in docs]
        lens = [len(s) for d in docs for s in d]
        tok = [t for d in docs for s in d for t in sorted(s)]
        return Corpus(_csr(np.asarray(sizes, np.int64)), _csr(np.asarray(lens, np.int64)),
                      np.asarray(tok, np.int32))
    k = [len(set(l)) for l in dic_lists]
    off = _csr(np.asarray(k, np.int64)).astype(np.int32)
    tgt = np.asarray([t for l in dic_lists for t in sorted(set(l))], np.int32)
    vt = v_tgt if v_tgt is not None else (int(tgt.max()) + 1 if len(tgt) else 1)
    for d in tgt_docs:
        for s in d:
            if len(s):
                vt = max(vt, max(s) + 1)
    dic = Dictionary(len(dic_lists), vt, off, tgt)
    n = len(src_docs)
    return Batch(corpus(src_docs), corpus(tgt_docs), dic, np.zeros(n, bool),
                 [np.zeros((0, 2), np.int32) for _ in range(n)])


@dataclass
class Anchors:
    """Per-sentence anchor ids (CSR over the sentences of one corpus): the
    language-independent names, dates, numbers and reference keys a sentence
    carries, ids in [0, v_anchor), sorted and distinct per sentence."""
    sent_off: np.ndarray  # int64, n_sents+1
    ids: np.ndarray       # int32


def make_anchors(batch: Batch, seed: int, v_anchor: int = 100_000, p_anchor: float = 0.3,
                 p_keep: float = 0.9, max_per: int = 2) -> tuple:
    """Anchors for both corpora of a batch: a source sentence carries 1..max_per
    random anchors with probability p_anchor; the target sentence planted from
    it (its gold link) carries each of them with probability p_keep; every
    other target sentence carries random anchors like a source sentence.
    Returns (source Anchors, target Anchors)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def draw(n_sents):
        has = rng.random(n_sents) < p_anchor
        cnt = np.where(has, rng.integers(1, max_per + 1, n_sents), 0)
        return [sorted(set(rng.integers(0, v_anchor, int(c)).tolist())) for c in cnt]

    n_src = int(batch.src.sent_tok_off.size - 1)
    n_tgt = int(batch.tgt.sent_tok_off.size - 1)
    src = draw(n_src)
    tgt = draw(n_tgt)
    for k, g in enumerate(batch.gold):
        s0, t0 = int(batch.src.doc_sent_off[k]), int(batch.tgt.doc_sent_off[k])
        for i, j in np.asarray(g).reshape(-1, 2).tolist():
            kept = [a for a in src[s0 + i] if rng.random() < p_keep]
            tgt[t0 + j] = sorted(kept)

    def csr(lists):
        off = _csr(np.asarray([len(x) for x in lists], np.int64))
        ids = np.asarray([a for x in lists for a in x], np.int32)
        return Anchors(off, ids)
    return csr(src), csr(tgt)
