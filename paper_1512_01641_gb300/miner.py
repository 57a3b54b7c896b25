"""Python binding of libminer.so (include/miner.h): argument marshalling only.

Every step of the mining path runs in the library's CUDA kernels; this module
only passes torch CUDA tensors' device pointers and the current stream through
ctypes.  There is no CPU fallback: if the library is missing or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MINE_OK, MINE_EINVAL, MINE_ENOMEM, MINE_ECUDA, MINE_ETIMEOUT, MINE_ENOTSUP = 0, -1, -2, -3, -4, -5
OPTIONS = {"tile_cols": 1, "tile_min_cells": 2, "tile_min_rows": 3, "wait_limit": 4, "link_recount": 5,
           "use_graph": 6, "graph_captures": 7, "fault_skip_flag": 8, "n_tile_flags": 9,
           "soft_split": 10, "fault_skip_soft": 11, "host_chunks": 12,
           "soft_split_q4": 13, "soft_order": 14}


class MinerError(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = _lib_or_none()
        msg = lib.mine_strerror(code).decode() if lib is not None else str(code)
        extra = ""
        if code == MINE_ECUDA and lib is not None:
            extra = f" (cudaError {lib.mine_last_cuda_error()})"
        super().__init__(f"{what}: {msg}{extra}")
        self.code = code


class _Corpus(C.Structure):
    _fields_ = [("n_docs", C.c_int64), ("n_sents", C.c_int64), ("n_tok", C.c_int64),
                ("doc_sent_off", C.c_void_p), ("sent_tok_off", C.c_void_p), ("tok", C.c_void_p)]


class _Dict(C.Structure):
    _fields_ = [("v_src", C.c_int32), ("v_tgt", C.c_int32), ("n_entries", C.c_int64),
                ("off", C.c_void_p), ("tgt", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("w", C.c_float * 4), ("b", C.c_float), ("gap", C.c_float), ("thr", C.c_float)]


class _SoftOpts(C.Structure):
    _fields_ = [("gamma", C.c_float), ("tau", C.c_float), ("eps", C.c_float), ("pairs", C.c_void_p),
                ("n_pairs", C.c_int64), ("n_cells", C.c_int64)]


class _Out(C.Structure):
    _fields_ = [("link_off", C.c_void_p), ("link_i", C.c_void_p), ("link_j", C.c_void_p),
                ("link_s", C.c_void_p), ("pair_score", C.c_void_p), ("link_capacity", C.c_int64)]


class _BiOut(C.Structure):
    _fields_ = [("link_off", C.c_void_p), ("link_i", C.c_void_p), ("link_j", C.c_void_p),
                ("s_fwd", C.c_void_p), ("s_rev", C.c_void_p), ("link_capacity", C.c_int64)]


# Every exported symbol of include/miner.h with its ctypes signature.
_SIGS = {
    "mine_plan_create": (C.c_int, [C.POINTER(_Corpus), C.POINTER(_Corpus), C.POINTER(_Dict),
                                   C.POINTER(C.c_void_p), C.c_void_p]),
    "mine_plan_create_with_options": (C.c_int, [C.POINTER(_Corpus), C.POINTER(_Corpus), C.POINTER(_Dict),
                                                C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.c_int,
                                                C.POINTER(C.c_void_p), C.c_void_p]),
    "mine_plan_destroy": (None, [C.c_void_p]),
    "mine_plan_n_pairs": (C.c_int64, [C.c_void_p]),
    "mine_plan_n_cells": (C.c_int64, [C.c_void_p]),
    "mine_plan_link_capacity": (C.c_int64, [C.c_void_p]),
    "mine_plan_cell_offsets": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mine_count": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mine_score": (C.c_int, [C.c_void_p, C.POINTER(_Params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mine_align": (C.c_int, [C.c_void_p, C.POINTER(_Params), C.c_void_p, C.POINTER(_Out), C.c_void_p]),
    "mine_pairs": (C.c_int, [C.c_void_p, C.POINTER(_Params), C.POINTER(_Out), C.c_void_p]),
    "mine_plan_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mine_link_gold_counts": (C.c_int, [C.c_void_p, C.POINTER(_Out), C.c_void_p, C.c_void_p, C.c_void_p]),
    "mine_dict_transpose": (C.c_int, [C.POINTER(_Dict), C.c_void_p, C.c_void_p, C.c_void_p]),
    "mine_corpus_add_anchors": (C.c_int, [C.POINTER(_Corpus), C.c_int32, C.c_void_p, C.c_void_p, C.c_int64,
                                          C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mine_dict_add_anchors": (C.c_int, [C.POINTER(_Dict), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mine_links_combine": (C.c_int, [C.c_void_p, C.POINTER(_Out), C.c_void_p, C.POINTER(_Out), C.c_int,
                                     C.POINTER(_BiOut), C.c_void_p]),
    "mine_plan_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int64]),
    "mine_plan_get_option": (C.c_int64, [C.c_void_p, C.c_int]),
    "mine_plan_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "mine_plan_kernel_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "softnw_workspace_size": (C.c_int64, [C.c_void_p]),
    "softnw_fwd": (C.c_int, [C.c_void_p, C.POINTER(_Params), C.POINTER(_SoftOpts), C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "softnw_bwd": (C.c_int, [C.c_void_p, C.POINTER(_Params), C.POINTER(_SoftOpts), C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mine_pairs_host": (C.c_int, [C.POINTER(_Corpus), C.POINTER(_Corpus), C.POINTER(_Dict), C.POINTER(_Params),
                                  C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int64, C.c_void_p]),
    "mine_unconstrained_workspace_size": (C.c_int64, [C.c_void_p]),
    "mine_unconstrained_link_capacity": (C.c_int64, [C.c_void_p]),
    "mine_align_unconstrained": (C.c_int, [C.c_void_p, C.POINTER(_Params), C.c_void_p, C.c_void_p, C.POINTER(_Out),
                                           C.c_void_p]),
    "mine_align_pair_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                         C.POINTER(_Params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p]),
    "mine_strerror": (C.c_char_p, [C.c_int]),
    "mine_last_cuda_error": (C.c_int, []),
}

_lib = None


def _lib_or_none():
    return _lib


def lib(build_if_missing: bool = False) -> C.CDLL:
    """Load libminer.so (raises if it is absent; never falls back)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libminer.so not built ({path}); run __graft_entry__.build()")
            _build.build()
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, what: str):
    if code != MINE_OK:
        raise MinerError(code, what)


@dataclass
class MineParams:
    """Classifier weights w (4) and bias b, gap penalty, acceptance threshold."""
    w: tuple = (4.0, 4.0, -2.0, 1.0)
    b: float = -3.0
    gap: float = 0.3
    thr: float = 0.5

    def c(self) -> _Params:
        p = _Params()
        for k in range(4):
            p.w[k] = float(self.w[k])
        p.b, p.gap, p.thr = float(self.b), float(self.gap), float(self.thr)
        return p


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


class DeviceBatch:
    """Corpus pair and dictionary resident on the GPU (int64 offsets, int32 ids)."""

    def __init__(self, src_doc, src_sent, src_tok, tgt_doc, tgt_sent, tgt_tok, dict_off, dict_tgt,
                 v_src: int, v_tgt: int):
        self.src = (src_doc, src_sent, src_tok)
        self.tgt = (tgt_doc, tgt_sent, tgt_tok)
        self.dict_off, self.dict_tgt = dict_off, dict_tgt
        self.v_src, self.v_tgt = int(v_src), int(v_tgt)

    @classmethod
    def from_batch(cls, batch, device="cuda", non_blocking=False):
        import torch

        def up(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
            return t.to(device, non_blocking=non_blocking)
        return cls(up(batch.src.doc_sent_off, np.int64), up(batch.src.sent_tok_off, np.int64),
                   up(batch.src.tok, np.int32), up(batch.tgt.doc_sent_off, np.int64),
                   up(batch.tgt.sent_tok_off, np.int64), up(batch.tgt.tok, np.int32),
                   up(batch.dic.off, np.int32), up(batch.dic.tgt, np.int32), batch.dic.v_src, batch.dic.v_tgt)

    def reversed(self, dict_off=None, dict_tgt=None, stream=None) -> "DeviceBatch":
        """The same pairs with the roles swapped (target documents become the
        source), for mining the reverse direction; its dictionary maps this
        batch's target ids to source ids: the given CSR (dict_off: v_tgt+1,
        dict_tgt), or the transpose of this batch's dictionary."""
        if dict_off is None:
            dict_off, dict_tgt = dict_transpose(self.dict_off, self.dict_tgt, self.v_src, self.v_tgt, stream)
        return DeviceBatch(*self.tgt, *self.src, dict_off, dict_tgt, self.v_tgt, self.v_src)

    def c_structs(self):
        def corpus(doc, sent, tok):
            c = _Corpus()
            c.n_docs = doc.numel() - 1
            c.n_sents = sent.numel() - 1
            c.n_tok = tok.numel()
            c.doc_sent_off, c.sent_tok_off, c.tok = doc.data_ptr(), sent.data_ptr(), tok.data_ptr() if tok.numel() else 0
            return c
        d = _Dict()
        d.v_src, d.v_tgt = self.v_src, self.v_tgt
        d.n_entries = self.dict_tgt.numel()
        d.off, d.tgt = self.dict_off.data_ptr(), self.dict_tgt.data_ptr() if self.dict_tgt.numel() else 0
        return corpus(*self.src), corpus(*self.tgt), d


class Plan:
    """A mining plan (mine_plan_create) over a DeviceBatch.  options: plan
    options by OPTIONS name, set before the work lists are built
    (mine_plan_create_with_options)."""

    def __init__(self, dbatch: DeviceBatch, stream=None, options: dict | None = None):
        L = lib()
        self.dbatch = dbatch  # keeps the inputs alive
        self._src, self._tgt, self._dict = dbatch.c_structs()
        h = C.c_void_p()
        opts = dict(options or {})
        ids = (C.c_int32 * max(len(opts), 1))(*[OPTIONS[k] for k in opts])
        vals = (C.c_int64 * max(len(opts), 1))(*[int(v) for v in opts.values()])
        _check(L.mine_plan_create_with_options(C.byref(self._src), C.byref(self._tgt), C.byref(self._dict), ids,
                                               vals, len(opts), C.byref(h), _stream(stream)),
               "mine_plan_create_with_options")
        self._h = h
        self.n_pairs = L.mine_plan_n_pairs(h)
        self.n_cells = L.mine_plan_n_cells(h)
        self.link_capacity = L.mine_plan_link_capacity(h)
        off = np.zeros(self.n_pairs + 1, np.int64)
        _check(L.mine_plan_cell_offsets(h, off.ctypes.data), "mine_plan_cell_offsets")
        self.cell_offsets = off

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().mine_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    KERNEL_KINDS = ("count", "fill", "walk", "links", "scan", "score", "soft_fwd", "soft_bwd")

    def set_option(self, name: str, value: int):
        _check(lib().mine_plan_set_option(self._h, OPTIONS[name], int(value)), f"mine_plan_set_option({name})")

    def get_option(self, name: str) -> int:
        return int(lib().mine_plan_get_option(self._h, OPTIONS[name]))

    def check(self, stream=None):
        """Synchronise and raise if a device-side wait timed out (mine_plan_check)."""
        _check(lib().mine_plan_check(self._h, _stream(stream)), "mine_plan_check")

    def set_timing(self, enable: bool = True):
        _check(lib().mine_plan_set_timing(self._h, int(enable)), "mine_plan_set_timing")

    def kernel_times(self):
        """{kind: (total ms, launches)} of the launches since set_timing(True)."""
        n = len(self.KERNEL_KINDS)
        ms = np.zeros(n, np.float32)
        cnt = np.zeros(n, np.int64)
        r = lib().mine_plan_kernel_times(self._h, ms.ctypes.data, cnt.ctypes.data, n)
        if r < 0:
            _check(r, "mine_plan_kernel_times")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KERNEL_KINDS)}

    # ------------------------------------------------------------------ calls
    def count(self, out=None, stream=None):
        """(n_cells, 2) uint8 tensor of (ms, mt) per cell."""
        import torch
        if out is None:
            out = torch.empty((self.n_cells, 2), dtype=torch.uint8, device="cuda")
        _check(lib().mine_count(self._h, _ptr(out), _stream(stream)), "mine_count")
        return out

    def score(self, params: MineParams, counts, want_features=False, stream=None):
        import torch
        s = torch.empty(self.n_cells, dtype=torch.float32, device="cuda")
        f = torch.empty((self.n_cells, 4), dtype=torch.float32, device="cuda") if want_features else None
        p = params.c()
        _check(lib().mine_score(self._h, C.byref(p), _ptr(counts), _ptr(s), _ptr(f), _stream(stream)), "mine_score")
        return (s, f) if want_features else s

    def new_output(self):
        import torch
        cap = max(self.link_capacity, 1)
        return {
            "link_off": torch.empty(self.n_pairs + 1, dtype=torch.int64, device="cuda"),
            "link_i": torch.empty(cap, dtype=torch.int32, device="cuda"),
            "link_j": torch.empty(cap, dtype=torch.int32, device="cuda"),
            "link_s": torch.empty(cap, dtype=torch.float32, device="cuda"),
            "pair_score": torch.empty(max(self.n_pairs, 1), dtype=torch.float32, device="cuda"),
        }

    @staticmethod
    def _out_struct(o, cap):
        s = _Out()
        s.link_off = o["link_off"].data_ptr()
        s.link_i, s.link_j, s.link_s = o["link_i"].data_ptr(), o["link_j"].data_ptr(), o["link_s"].data_ptr()
        s.pair_score = o["pair_score"].data_ptr()
        s.link_capacity = cap
        return s

    def align(self, params: MineParams, counts, out=None, stream=None):
        out = out if out is not None else self.new_output()
        s = self._out_struct(out, out["link_i"].numel())
        p = params.c()
        _check(lib().mine_align(self._h, C.byref(p), _ptr(counts), C.byref(s), _stream(stream)), "mine_align")
        return out

    def link_gold_counts(self, out, gold, stream=None):
        """(links that are gold, links, gold cells) of an alignment output."""
        import torch
        res = torch.zeros(3, dtype=torch.int64, device="cuda")
        s = self._out_struct(out, out["link_i"].numel())
        _check(lib().mine_link_gold_counts(self._h, C.byref(s), _ptr(gold), _ptr(res), _stream(stream)),
               "mine_link_gold_counts")
        return res

    def align_unconstrained(self, params: MineParams, counts, out=None, ws=None, stream=None):
        """The unconstrained (Yalign A*) aligner from counts
        (mine_align_unconstrained): per pair the matched cells with s >= thr
        in source order and the FP64 score."""
        import torch
        L = lib()
        cap = max(int(L.mine_unconstrained_link_capacity(self._h)), 1)
        if out is None:
            out = {"link_off": torch.empty(self.n_pairs + 1, dtype=torch.int64, device="cuda"),
                   "link_i": torch.empty(cap, dtype=torch.int32, device="cuda"),
                   "link_j": torch.empty(cap, dtype=torch.int32, device="cuda"),
                   "link_s": torch.empty(cap, dtype=torch.float32, device="cuda"),
                   "pair_score": torch.empty(max(self.n_pairs, 1), dtype=torch.float32, device="cuda")}
        if ws is None:
            ws = torch.empty(int(L.mine_unconstrained_workspace_size(self._h)), dtype=torch.uint8, device="cuda")
        s = self._out_struct(out, out["link_i"].numel())
        p = params.c()
        _check(L.mine_align_unconstrained(self._h, C.byref(p), _ptr(counts), _ptr(ws), C.byref(s), _stream(stream)),
               "mine_align_unconstrained")
        out["_ws"] = ws
        return out

    def mine(self, params: MineParams, out=None, stream=None):
        """The whole hot path (counts, similarity, alignment, threshold)."""
        out = out if out is not None else self.new_output()
        s = self._out_struct(out, out["link_i"].numel())
        p = params.c()
        _check(lib().mine_pairs(self._h, C.byref(p), C.byref(s), _stream(stream)), "mine_pairs")
        return out


def dict_transpose(dict_off, dict_tgt, v_src: int, v_tgt: int, stream=None):
    """mine_dict_transpose: the CSR dictionary from target ids to the sorted
    source ids that translate to them -> (off: v_tgt+1 int32, tgt int32)."""
    import torch
    d = _Dict()
    d.v_src, d.v_tgt = int(v_src), int(v_tgt)
    d.n_entries = dict_tgt.numel()
    d.off, d.tgt = dict_off.data_ptr(), dict_tgt.data_ptr() if dict_tgt.numel() else 0
    off = torch.empty(int(v_tgt) + 1, dtype=torch.int32, device=dict_off.device)
    tgt = torch.empty(max(dict_tgt.numel(), 1), dtype=torch.int32, device=dict_off.device)
    _check(lib().mine_dict_transpose(C.byref(d), _ptr(off), _ptr(tgt), _stream(stream)), "mine_dict_transpose")
    return off, tgt[:dict_tgt.numel()]


def add_anchors(dbatch: DeviceBatch, src_anchors, tgt_anchors, v_anchor: int, stream=None) -> DeviceBatch:
    """Anchors (Section 5.3): the batch with every sentence's anchor ids
    (src_anchors / tgt_anchors: (sent_off int64, ids int32) device tensors,
    per sentence sorted and distinct, ids in [0, v_anchor)) among its tokens
    and the anchors' identity entries in the dictionary
    (mine_corpus_add_anchors, mine_dict_add_anchors)."""
    import torch
    L = lib()
    cs, ct, d = dbatch.c_structs()

    def corpus(c, words, anc, v_words):
        aoff, ids = anc
        off = torch.empty(words[1].numel(), dtype=torch.int64, device=words[1].device)
        tok = torch.empty(max(words[2].numel() + ids.numel(), 1), dtype=torch.int32, device=words[1].device)
        _check(L.mine_corpus_add_anchors(C.byref(c), int(v_words), _ptr(aoff), _ptr(ids), ids.numel(), int(v_anchor),
                                         _ptr(off), _ptr(tok), _stream(stream)), "mine_corpus_add_anchors")
        return words[0], off, tok[:words[2].numel() + ids.numel()]
    src = corpus(cs, dbatch.src, src_anchors, dbatch.v_src)
    tgt = corpus(ct, dbatch.tgt, tgt_anchors, dbatch.v_tgt)
    off = torch.empty(dbatch.v_src + v_anchor + 1, dtype=torch.int32, device=dbatch.dict_off.device)
    tgt_d = torch.empty(dbatch.dict_tgt.numel() + v_anchor, dtype=torch.int32, device=dbatch.dict_off.device)
    _check(L.mine_dict_add_anchors(C.byref(d), int(v_anchor), _ptr(off), _ptr(tgt_d), _stream(stream)),
           "mine_dict_add_anchors")
    return DeviceBatch(*src, *tgt, off, tgt_d, dbatch.v_src + v_anchor, dbatch.v_tgt + v_anchor)


BI_MODES = {"union": 0, "intersect": 1}


def combine_links(fwd: "Plan", out_fwd, rev: "Plan", out_rev, mode: str = "union", out=None, stream=None):
    """mine_links_combine: per pair, the union (or intersection) of the
    forward links and the reverse plan's links mapped back to forward
    coordinates -> dict of link_off, link_i, link_j, s_fwd, s_rev (NaN where a
    direction did not keep the link)."""
    import torch
    cap = max(fwd.link_capacity + rev.link_capacity, 1)
    if out is None:
        out = {"link_off": torch.empty(fwd.n_pairs + 1, dtype=torch.int64, device="cuda"),
               "link_i": torch.empty(cap, dtype=torch.int32, device="cuda"),
               "link_j": torch.empty(cap, dtype=torch.int32, device="cuda"),
               "s_fwd": torch.empty(cap, dtype=torch.float32, device="cuda"),
               "s_rev": torch.empty(cap, dtype=torch.float32, device="cuda")}
    b = _BiOut()
    b.link_off, b.link_i, b.link_j = (out[k].data_ptr() for k in ("link_off", "link_i", "link_j"))
    b.s_fwd, b.s_rev = out["s_fwd"].data_ptr(), out["s_rev"].data_ptr()
    b.link_capacity = out["link_i"].numel()
    f = Plan._out_struct(out_fwd, out_fwd["link_i"].numel())
    r = Plan._out_struct(out_rev, out_rev["link_i"].numel())
    _check(lib().mine_links_combine(fwd.handle, C.byref(f), rev.handle, C.byref(r), BI_MODES[mode], C.byref(b),
                                    _stream(stream)), "mine_links_combine")
    return out


class BiPlan:
    """Bi-directional mining (Section 5.4, BI): a forward plan over the batch
    and a reverse plan over its reversed view (corpora swapped, dictionary
    from target ids to source ids), mined with their own parameters; mine()
    returns both directions' outputs and their per-pair combination."""

    def __init__(self, dbatch: DeviceBatch, rev_dict=None, options: dict | None = None, stream=None):
        rd = rev_dict if rev_dict is not None else (None, None)
        self.fwd = Plan(dbatch, stream=stream, options=options)
        self.rev = Plan(dbatch.reversed(*rd, stream=stream), stream=stream, options=options)
        self.n_pairs = self.fwd.n_pairs

    def mine(self, params_fwd: MineParams, params_rev: MineParams, mode: str = "union", stream=None):
        of = self.fwd.mine(params_fwd, stream=stream)
        orv = self.rev.mine(params_rev, stream=stream)
        return of, orv, combine_links(self.fwd, of, self.rev, orv, mode, stream=stream)

    def close(self):
        self.fwd.close()
        self.rev.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def mine_host(host, v_src: int, v_tgt: int, params: "MineParams", options: dict | None = None, out=None,
              stream=None):
    """mine_pairs_host: the whole hot path from host arrays.  host: the eight
    CSR arrays (src doc/sent/tok, tgt doc/sent/tok, dict off/tgt) as numpy
    arrays or CPU tensors (pinned ones copy at full speed); out (optional):
    host tensors link_off, link_i, link_j, link_s, pair_score to fill.
    Returns out with the links of every pair."""
    import torch
    t = [x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x)) for x in host]
    n = t[0].numel() - 1
    ns, mt = torch.diff(t[0]), torch.diff(t[3])
    cap = max(int(torch.minimum(ns, mt).sum()), 1)
    if out is None:
        out = {"link_off": torch.empty(n + 1, dtype=torch.int64), "link_i": torch.empty(cap, dtype=torch.int32),
               "link_j": torch.empty(cap, dtype=torch.int32), "link_s": torch.empty(cap, dtype=torch.float32),
               "pair_score": torch.empty(max(n, 1), dtype=torch.float32)}

    def corpus(doc, sent, tok):
        c = _Corpus()
        c.n_docs, c.n_sents, c.n_tok = doc.numel() - 1, sent.numel() - 1, tok.numel()
        c.doc_sent_off, c.sent_tok_off, c.tok = doc.data_ptr(), sent.data_ptr(), tok.data_ptr() if tok.numel() else 0
        return c
    cs, ct = corpus(*t[0:3]), corpus(*t[3:6])
    d = _Dict()
    d.v_src, d.v_tgt, d.n_entries = int(v_src), int(v_tgt), t[7].numel()
    d.off, d.tgt = t[6].data_ptr(), t[7].data_ptr() if t[7].numel() else 0
    opts = dict(options or {})
    ids = (C.c_int32 * max(len(opts), 1))(*[OPTIONS[k] for k in opts])
    vals = (C.c_int64 * max(len(opts), 1))(*[int(v) for v in opts.values()])
    p = params.c()
    _check(lib().mine_pairs_host(C.byref(cs), C.byref(ct), C.byref(d), C.byref(p), ids, vals, len(opts),
                                 out["link_off"].data_ptr(), out["link_i"].data_ptr(), out["link_j"].data_ptr(),
                                 out["link_s"].data_ptr(), out["pair_score"].data_ptr(), out["link_i"].numel(),
                                 _stream(stream)), "mine_pairs_host")
    return out


def noalloc_result(n_links: int, pair_score: float):
    """The (n_links, pair_score) that mine_align_pair_noalloc wrote, checked:
    n_links == -1 (with a NaN score) says that a bounded wait for the staged
    counts gave up on the device, so the links are invalid -- raised as
    MINE_ETIMEOUT; anything else is returned unchanged."""
    if int(n_links) == -1:
        raise MinerError(MINE_ETIMEOUT, "mine_align_pair_noalloc (device-side staging wait)")
    if int(n_links) < 0:
        raise MinerError(MINE_EINVAL, f"mine_align_pair_noalloc: n_links = {int(n_links)}")
    return int(n_links), float(pair_score)


def links_per_pair(out, n_pairs):
    """Split a mining output (on any device) into per-pair lists of (i, j, s)."""
    off = out["link_off"].cpu().numpy()
    li, lj, ls = (out[k].cpu().numpy() for k in ("link_i", "link_j", "link_s"))
    return [list(zip(li[off[k]:off[k + 1]].tolist(), lj[off[k]:off[k + 1]].tolist(),
                     ls[off[k]:off[k + 1]].tolist())) for k in range(n_pairs)]


# ---------------------------------------------------------------------------
# soft alignment (softnw_fwd / softnw_bwd) and its autograd wrapper
# ---------------------------------------------------------------------------
THETA_NAMES = ("w0", "w1", "w2", "w3", "b", "gap", "thr")


def params_from_theta(theta) -> MineParams:
    t = [float(x) for x in theta]
    return MineParams(w=tuple(t[:4]), b=t[4], gap=t[5], thr=t[6])


class SoftAligner:
    """Soft alignment loss over a plan's pairs, from cached counts and gold
    links (one 0/1 byte per cell, row-major per pair like the counts)."""

    def __init__(self, plan: Plan, counts, gold, gamma: float, tau: float = 0.05, eps: float = 1e-7):
        import torch
        self.plan, self.counts, self.gold = plan, counts, gold
        self.opts = _SoftOpts(float(gamma), float(tau), float(eps), None, 0, 0)
        self._sel = None
        n = lib().softnw_workspace_size(plan.handle)
        if n < 0:
            _check(int(n), "softnw_workspace_size")
        self.ws = torch.empty(max(int(n), 1), dtype=torch.uint8, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.grad = torch.zeros(7, dtype=torch.float32, device="cuda")

    def select(self, pairs=None):
        """Restrict the next forward/backward to these pairs (a minibatch;
        host indices, or None for all pairs); the loss is their cells' mean."""
        import torch
        if pairs is None:
            self._sel = None
            self.opts.pairs, self.opts.n_pairs, self.opts.n_cells = None, 0, 0
            return
        pairs = np.asarray(pairs, np.int32)
        sizes = np.diff(self.plan.cell_offsets)[pairs]
        pairs = pairs[np.argsort(-sizes, kind="stable")]  # largest first (load balance)
        self._sel = torch.from_numpy(pairs).cuda()
        self.opts.pairs = self._sel.data_ptr()
        self.opts.n_pairs = len(pairs)
        self.opts.n_cells = int(sizes.sum())

    def forward(self, params: MineParams, want_value=False, want_expected=False, stream=None):
        import torch
        value = torch.empty(max(self.plan.n_pairs, 1), dtype=torch.float32, device="cuda") if want_value else None
        exp = torch.empty(max(self.plan.n_cells, 1), dtype=torch.float32, device="cuda") if want_expected else None
        p = params.c()
        _check(lib().softnw_fwd(self.plan.handle, C.byref(p), C.byref(self.opts), _ptr(self.counts), _ptr(self.gold),
                                _ptr(self.ws), _ptr(self.loss), _ptr(value), _ptr(exp), _stream(stream)), "softnw_fwd")
        return self.loss, value, exp

    def backward(self, params: MineParams, dloss: float = 1.0, want_hvp=False, stream=None):
        import torch
        hvp = torch.empty(max(self.plan.n_cells, 1), dtype=torch.float32, device="cuda") if want_hvp else None
        p = params.c()
        _check(lib().softnw_bwd(self.plan.handle, C.byref(p), C.byref(self.opts), _ptr(self.counts), _ptr(self.gold),
                                _ptr(self.ws), C.c_float(dloss), _ptr(self.grad), _ptr(hvp), _stream(stream)),
               "softnw_bwd")
        return (self.grad, hvp) if want_hvp else self.grad


def _soft_fn():
    import torch

    class SoftNWLoss(torch.autograd.Function):
        """loss = SoftNWLoss.apply(theta, aligner), theta = [w0..w3, b, gap, thr].

        Forward and backward run in the library's kernels (softnw_fwd /
        softnw_bwd); theta is read back to the host for the kernel arguments."""

        @staticmethod
        def forward(ctx, theta, aligner):
            params = params_from_theta(theta.detach().cpu().tolist())
            loss, _, _ = aligner.forward(params)
            ctx.aligner, ctx.params = aligner, params
            return loss[0].clone()

        @staticmethod
        def backward(ctx, dloss):
            g = ctx.aligner.backward(ctx.params, float(dloss))
            return g.clone().to(dloss.dtype), None

    return SoftNWLoss


_SOFT_FN = None


def soft_nw_loss(theta, aligner: SoftAligner):
    """Differentiable soft-alignment loss (autograd through the CUDA kernels)."""
    global _SOFT_FN
    if _SOFT_FN is None:
        _SOFT_FN = _soft_fn()
    return _SOFT_FN.apply(theta, aligner)


def gold_cells(batch, plan: Plan):
    """One 0/1 byte per cell from the batch's planted gold links (host array)."""
    g = np.zeros(max(plan.n_cells, 1), np.uint8)
    M = batch.tgt.doc_sizes()
    for k, links in enumerate(batch.gold):
        if len(links):
            g[plan.cell_offsets[k] + links[:, 0].astype(np.int64) * M[k] + links[:, 1]] = 1
    return g
