#!/usr/bin/env python
"""Benchmark of the batched mining hot path on GB300.

Workload (default): the large uneven batch -- 100,000 Wikipedia-shaped
document pairs (lognormal sentence counts, median 60, sigma 0.8, clipped
5..800, half planted) plus 8 pairs of 5,000 x 5,000 sentences, all in one
plan; sentences of 5..30 Zipf(1.1) token ids over 50k-id vocabularies.  One
step = one mine_pairs call over the whole batch: overlap counts, similarity,
Needleman-Wunsch fill, traceback + threshold, link compaction.

Prints one JSON line (rank 0).  ``value`` is DP cell-updates per second over
all ranks (sum over pairs of N*M per step), inputs resident in HBM;
``e2e`` is the same metric through the public API from pinned host buffers
(upload, plan, mine, download of links and scores inside the timed region).

--impl reference times the FP64 CPU oracle (the correctness reference) on a
bounded random sample of the same workload, on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from paper_1512_01641_gb300 import synth  # noqa: E402

METRIC = "DP cell-updates/s (batched hard-NW mining)"
UNIT = "cell-updates/s"
LANES_PER_SM = 128  # issue model: 4 sub-partitions x one 32-lane warp instruction per clock
PEAKS = os.path.join(HERE, "MEASURED_PEAKS.json")
TUNE_DICT_DROP = 0.3   # share of dictionary entries the miner does not know (tuning and BI records)
TUNE_THETA0 = [4.0, 4.0, -2.0, 1.0, -6.0, 0.8, 0.8]  # poor start: b, gap, thr at the grid's far corner
HBM_FALLBACK_GBS = 6800.0  # one earlier GB300 copy measurement, used only without MEASURED_PEAKS.json
# algorithmic lane-operations per cell of the roofline model when the path is
# timed from precomputed counts (similarity and DP only)
OPS_SIM = 11   # 4 quotients, 4 multiply-adds, exp, add, reciprocal
OPS_DP = 8     # 3 candidates, 2 max, 2 compare/select, 1 pack


# DRAM bytes per cell of the dominant kernels, from one ncu capture
# (profiles/), valid only while the kernel's source is unchanged.
TRAFFIC = {
    "count": {"file": "paper_1512_01641_gb300/csrc/count.cu", "sha1": "0aedd7dcb9d2b315a125ae74fa594893687bcc88",
              "bytes_per_cell": (260.129792e6 + 467.148544e6) / 218470577},
}


def traffic_per_launch(kind, cells):
    import hashlib
    t = TRAFFIC.get(kind)
    if not t or not t["sha1"] or t["bytes_per_cell"] is None:
        return None
    try:
        with open(os.path.join(HERE, t["file"]), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != t["sha1"]:
                return None
    except OSError:
        return None
    return t["bytes_per_cell"] * cells


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--pairs", type=int, default=100_000, help="Wikipedia-shaped pairs per rank")
    ap.add_argument("--long", type=int, default=8, help="5000x5000 pairs per rank")
    ap.add_argument("--long-n", type=int, default=5000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-stream-steps", type=int, default=16)
    ap.add_argument("--cpu-pairs", type=int, default=8000, help="pairs in the oracle's timed sample")
    ap.add_argument("--no-tune", action="store_true", help="skip the tuning comparison")
    ap.add_argument("--tune-pairs", type=int, default=50_000)
    ap.add_argument("--tune-eval", type=int, default=10_000)
    ap.add_argument("--tune-steps", type=int, default=200)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-bi", action="store_true", help="skip the bi-directional mining record")
    ap.add_argument("--no-anchors", action="store_true", help="skip the anchor-token record")
    ap.add_argument("--bi-pairs", type=int, default=10_000)
    ap.add_argument("--anchor-pairs", type=int, default=10_000)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-pair, 10,000-pair, NW-only and soft-NW records")
    ap.add_argument("--soft-step", action="store_true",
                    help="only time one soft-NW forward+backward (profiling): on a 4,096-pair tuning minibatch, "
                         "or with --soft-config soft on the 4,096 planted pairs of the soft configuration")
    ap.add_argument("--soft-config", default="tune", choices=["tune", "soft"])
    ap.add_argument("--soft-pairs", type=int, default=4096, help="pairs of the --soft-step minibatch")
    return ap.parse_args()


def dist_env():
    r = int(os.environ.get("RANK", 0))
    w = int(os.environ.get("WORLD_SIZE", 1))
    lr = int(os.environ.get("LOCAL_RANK", 0))
    return r, w, lr


def workload(args, rank):
    b = synth.uneven_batch(n_pairs=args.pairs, n_long=args.long, long_n=args.long_n,
                           seed=synth.SEED_BASE + 2 + 1000 * rank)
    desc = {"workload": f"uneven batch: {args.pairs} Wikipedia-shaped pairs + {args.long} x "
                        f"{args.long_n}x{args.long_n} pairs per GPU",
            "pairs_per_gpu": b.n_pairs, "cells_per_gpu": b.cells(),
            "tokens_per_gpu": int(len(b.src.tok) + len(b.tgt.tok)),
            "params": {"w": [4, 4, -2, 1], "b": -3, "gap": 0.3, "thr": 0.5},
            "l2": "inputs larger than L2 (no flush)"}
    return b, desc


def merge_compare_ops(batch):
    """Sum over cells of |T_i| + lt_j: the compares of a sorted-merge intersection
    of source sentence i's translations with target sentence j."""
    dic = batch.dic
    fan = np.diff(dic.off.astype(np.int64))
    tr_per_tok = fan[batch.src.tok]
    s_off = batch.src.sent_tok_off
    tr_per_sent = np.add.reduceat(tr_per_tok, s_off[:-1]) if len(tr_per_tok) else np.zeros(0)
    d_off = batch.src.doc_sent_off
    n_src = np.diff(d_off)
    t_len = np.diff(batch.tgt.sent_tok_off)
    tr_doc = np.add.reduceat(np.append(tr_per_sent, 0), d_off[:-1])[: batch.n_pairs] * (n_src > 0)
    tl_doc = np.add.reduceat(np.append(t_len, 0), batch.tgt.doc_sent_off[:-1])[: batch.n_pairs] * \
        (np.diff(batch.tgt.doc_sent_off) > 0)
    M = np.diff(batch.tgt.doc_sent_off)
    return int((tr_doc * M + tl_doc * n_src).sum())


def sm_count():
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def hbm_peak():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def algorithmic_bytes(batch, n_links):
    """Bytes the method itself must move per step: the inputs once (corpora
    CSR and dictionary), the 2-bit traceback mask of every cell written once,
    the outputs once (12 bytes per link, a score and a link offset per pair).
    The count buffer between the count and fill kernels is a design choice,
    not counted."""
    src, tgt, dic = batch.src, batch.tgt, batch.dic
    inp = sum(a.nbytes for a in (src.doc_sent_off, src.sent_tok_off, src.tok, tgt.doc_sent_off,
                                 tgt.sent_tok_off, tgt.tok, dic.off, dic.tgt))
    cells = batch.cells()
    return inp + cells // 4 + 12 * n_links + 12 * batch.n_pairs


def timed_steps(fn, steps, warmup):
    """CUDA-event time (s) of `steps` calls of fn after `warmup` calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1000.0


def oracle_rate(batch, n_pairs=None, seed=0):
    """The FP64 oracle's cell-updates/s on (a sample of) a batch, all host cores."""
    import oracle
    pick = np.arange(batch.n_pairs)
    if n_pairs is not None and n_pairs < batch.n_pairs:
        pick = np.sort(np.random.default_rng(seed).choice(batch.n_pairs, n_pairs, replace=False))
    sub = batch.subset(pick)
    t0 = time.perf_counter()
    r = oracle.mine(sub, [4, 4, -2, 1], -3.0, 0.3, 0.5, n_threads=os.cpu_count() or 1)
    dt = time.perf_counter() - t0
    return {"value": sub.cells() / dt, "unit": UNIT, "cores": int(r["threads"]), "kind": "oracle",
            "sample": f"{len(pick)} pairs, {sub.cells()} cells, {dt:.2f} s"}


def config_records(args, params):
    """The other configurations of the benchmark spec, each with the oracle beside it:
    one 40 x 45 pair (latency of one call), 10,000 Wikipedia-shaped pairs
    (throughput), the NW-only rate of the bench batch's counts, and the soft
    alignment of 4,096 planted pairs at three temperatures."""
    import torch
    from paper_1512_01641_gb300 import miner
    rec = {}
    # single pair, 40 x 45: the latency of one mine_pairs call (graph replay)
    b1 = synth.single_pair()
    with miner.Plan(miner.DeviceBatch.from_batch(b1)) as plan:
        out = plan.mine(params)
        for _ in range(10):
            plan.mine(params, out)
        torch.cuda.synchronize()
        lat = []
        for _ in range(200):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.mine(params, out)
            b.record()
            torch.cuda.synchronize()
            lat.append(a.elapsed_time(b))
        host = []
        for _ in range(50):
            t0 = time.perf_counter()
            plan.mine(params, out)
            n = int(out["link_off"][-1].item())
            out["link_i"][:n].cpu()
            host.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    import oracle
    for _ in range(20):
        oracle.mine(b1, [4, 4, -2, 1], -3.0, 0.3, 0.5, n_threads=1)
    o1 = (time.perf_counter() - t0) / 20
    rec["single_pair_40x45"] = {"device_ms_median": float(np.median(lat)), "device_ms_p99": float(np.percentile(lat, 99)),
                                "call_and_readback_ms_median": 1000 * float(np.median(host)),
                                "cells": b1.cells(), "oracle_ms_one_core": 1000 * o1,
                                "timing": "CUDA events around each of 200 mine_pairs calls (graph replay)"}
    # 10,000 Wikipedia-shaped pairs
    b2 = synth.wiki_batch()
    with miner.Plan(miner.DeviceBatch.from_batch(b2)) as plan:
        out = plan.new_output()
        secs = timed_steps(lambda: plan.mine(params, out), args.steps, args.warmup)
        rec["wiki_10000"] = {"value": plan.n_cells * args.steps / secs, "unit": UNIT,
                             "pairs_per_s": plan.n_pairs * args.steps / secs, "ms_per_step": 1000 * secs / args.steps,
                             "cells": plan.n_cells, "oracle": oracle_rate(b2, 2000)}
    # the unconstrained (Yalign A*) aligner against Needleman-Wunsch on the
    # same 10,000 pairs: links, micro precision / recall against the planted
    # gold links, target sentences aligned more than once, and time
    with miner.Plan(miner.DeviceBatch.from_batch(b2)) as plan:
        counts = plan.count()
        gold = torch.from_numpy(miner.gold_cells(b2, plan)).cuda()
        res = {}
        for name in ("nw", "unconstrained"):
            run = (lambda: plan.align(params, counts)) if name == "nw" else \
                (lambda: plan.align_unconstrained(params, counts))
            o = run()
            secs = timed_steps(run, 3, 1)
            tp, nl, ng = (int(x) for x in plan.link_gold_counts(o, gold).cpu().tolist())
            links = miner.links_per_pair(o, b2.n_pairs)
            rep = sum(len(l) - len({j for _, j, _ in l}) for l in links)
            prec, rec_ = tp / max(nl, 1), tp / max(ng, 1)
            res[name] = {"links": nl, "correct": tp, "gold": ng, "precision": prec, "recall": rec_,
                         "f1": 2 * prec * rec_ / max(prec + rec_, 1e-12), "repeated_targets": rep,
                         "ms": 1000 * secs / 3}
        rec["unconstrained_vs_nw"] = {"pairs": b2.n_pairs, **res,
                                      "note": "same counts and classifier; the unconstrained aligner may move back "
                                              "into the target sequence (one gap penalty), so a target sentence "
                                              "can be aligned twice"}
    # soft alignment of 4,096 planted pairs of ~100 x 100 sentences
    b4 = synth.soft_batch()
    with miner.Plan(miner.DeviceBatch.from_batch(b4)) as plan:
        counts = plan.count()
        gold = torch.from_numpy(miner.gold_cells(b4, plan)).cuda()
        p = miner.params_from_theta([4.0, 4.0, -2.0, 1.0, -3.0, 0.3, 0.5])
        soft = {}
        for g in (1.0, 0.1, 0.01):
            al = miner.SoftAligner(plan, counts, gold, g, 0.05)
            tf = timed_steps(lambda: al.forward(p), args.steps, max(args.warmup, 2))
            tb = timed_steps(lambda: al.backward(p), args.steps, max(args.warmup, 2))
            soft[str(g)] = {"forward_ms": 1000 * tf / args.steps, "backward_ms": 1000 * tb / args.steps,
                            "cells_per_s_fwd_bwd": plan.n_cells * args.steps / (tf + tb)}
        plan.check()
        rec["soft_4096"] = {"pairs": plan.n_pairs, "cells": plan.n_cells, "tau": 0.05, "gamma": soft}
    return rec


def near_tie_record(batch, out_all, pick, ref, p_gap):
    """GPU paths (threshold off) against the oracle's (ref: oracle.mine of the
    pairs `pick`, the CPU sample) : identical diagonal sets, or a near tie (the
    GPU path re-scored in FP64 by the oracle within 1e-4 of the optimum), or a
    violation."""
    import oracle
    from paper_1512_01641_gb300 import miner
    links = miner.links_per_pair(out_all, batch.n_pairs)
    score = out_all["pair_score"].cpu().numpy()
    sub = batch.subset(pick)
    diff = []
    max_rel = 0.0
    for x, k in enumerate(pick):
        h = ref["score"][x]
        max_rel = max(max_rel, abs(float(score[k]) - h) / max(1.0, abs(h)))
        if [(i, j) for i, j, _ in links[k]] != [(i, j) for i, j, _ in ref["diag"][x]]:
            diff.append(x)
    ties = viol = 0
    if diff:
        rs = oracle.mine(sub.subset(diff), [4, 4, -2, 1], -3.0, p_gap, -1.0, want_sim=True)
        for y, x in enumerate(diff):
            got = oracle.path_score(rs["sim"][y], p_gap, [(i, j) for i, j, _ in links[pick[x]]])
            if got >= rs["score"][y] - 1e-4:
                ties += 1
            else:
                viol += 1
    return {"pairs_compared": len(pick), "paths_identical": len(pick) - len(diff), "near_ties": ties,
            "violations": viol, "max_pair_score_rel_err": max_rel,
            "rule": "GPU path (threshold off) vs oracle path; a differing path counts as a near tie when its FP64 "
                    "score is within 1e-4 of the optimum, else as a violation"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            time.sleep(0.3)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(batch, n_pairs, seed=0):
    import oracle
    rng = np.random.default_rng(seed)
    small = np.nonzero(batch.src.doc_sizes() * batch.tgt.doc_sizes() < 1_000_000)[0]
    pick = np.sort(rng.choice(small, size=min(n_pairs, len(small)), replace=False))
    sub = batch.subset(pick)
    cells = sub.cells()
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.mine(sub, [4, 4, -2, 1], -3.0, 0.3, 0.5, n_threads=threads)
    dt = time.perf_counter() - t0
    return {"value": cells / dt, "unit": UNIT, "cores": int(r["threads"]), "kind": "oracle",
            "sample": f"{len(pick)} random pairs of the workload (long pairs excluded), {cells} cells, "
                      f"{dt:.1f} s", "seconds": dt, "cells": cells}, pick, r


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    batch, desc = workload(args, 0)
    rng = np.random.default_rng(1)
    vals = []
    threads = os.cpu_count() or 1
    per_step = max(1, args.cpu_pairs // 4)
    import oracle
    small = np.nonzero(batch.src.doc_sizes() * batch.tgt.doc_sizes() < 1_000_000)[0]
    tot_cells = tot_t = 0.0
    for step in range(args.warmup + args.steps):
        pick = np.sort(rng.choice(small, size=min(per_step, len(small)), replace=False))
        sub = batch.subset(pick)
        t0 = time.perf_counter()
        oracle.mine(sub, [4, 4, -2, 1], -3.0, 0.3, 0.5, n_threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            tot_cells += sub.cells()
            tot_t += dt
    v = tot_cells / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": desc,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step {per_step} random pairs of the workload (long pairs excluded)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def soft_step(args):
    """One soft-NW forward + backward (the unit of an Adam step) on 4,096
    planted pairs of the tuning batch, after two warm-up passes; prints one
    JSON line with the CUDA-event times."""
    import torch
    from paper_1512_01641_gb300 import miner, tune
    if args.soft_config == "soft":
        td = tune.TuneData(synth.soft_batch(args.soft_pairs))
    else:
        rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 40))
        dic = synth.make_dictionary(rng, 50_000, 50_000)
        td = tune.TuneData(synth.tune_batch(args.soft_pairs, seed=synth.SEED_BASE + 4, dic=dic))
    al = miner.SoftAligner(td.plan, td.counts, td.gold, 0.1, 0.05)
    p = miner.params_from_theta(tune.THETA0)
    for _ in range(max(args.warmup, 2)):
        al.forward(p)
        al.backward(p)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    al.forward(p)
    ev[1].record()
    al.backward(p)
    ev[2].record()
    torch.cuda.synchronize()
    print(json.dumps({"soft_step": {"config": args.soft_config, "pairs": td.plan.n_pairs, "cells": td.plan.n_cells,
                                    "gamma": 0.1,
                                    "forward_ms": ev[0].elapsed_time(ev[1]),
                                    "backward_ms": ev[1].elapsed_time(ev[2])}}))


def run_tune(args):
    """Soft-NW gradient tuning (Adam) vs the 7^3 grid search and the paper's
    random search (343 draws), same GPU, evaluated by hard-NW micro-F1 on
    held-out planted pairs."""
    import dataclasses
    from paper_1512_01641_gb300 import tune
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 40))
    dic = synth.make_dictionary(rng, 50_000, 50_000)
    tr = synth.tune_batch(args.tune_pairs, seed=synth.SEED_BASE + 4, dic=dic)
    ev = synth.tune_batch(args.tune_eval, seed=synth.SEED_BASE + 5, dic=dic)
    # the planted data come from the full dictionary; the miner knows 70 % of
    # its entries, and every tuner starts from a poor setting
    thin = synth.thin_dictionary(dic, TUNE_DICT_DROP, synth.SEED_BASE + 41)
    tr, ev = dataclasses.replace(tr, dic=thin), dataclasses.replace(ev, dic=thin)
    r = tune.compare(tr, ev, steps=args.tune_steps, theta0=TUNE_THETA0)
    r["train_cells"] = tr.cells()
    r["mining_dictionary"] = f"{100 * (1 - TUNE_DICT_DROP):.0f} % of the planting dictionary's entries"
    return r


def run_bi(args, params, options):
    """Bi-directional mining (Section 5.4, BI) of 10,000 Wikipedia-shaped pairs
    (half planted): each direction has its own incomplete dictionary -- the
    forward one and the transpose of the planting dictionary, each missing an
    independent 30 % of its entries, as two separately trained phrase tables
    would -- and the reverse direction the mirrored classifier (the two
    overlap weights exchanged).  Links of each direction, their union and
    intersection against the gold links; device-timed steps of forward mining
    + reverse mining + union."""
    import dataclasses
    import torch
    from paper_1512_01641_gb300 import miner
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 50))
    dic = synth.make_dictionary(rng, 50_000, 50_000)
    b = synth.make_batch(synth.SEED_BASE + 51, args.bi_pairs, dic=dic)
    fwd_dic = synth.thin_dictionary(dic, TUNE_DICT_DROP, synth.SEED_BASE + 52)
    t_off, t_tgt = miner.dict_transpose(torch.from_numpy(dic.off).cuda(), torch.from_numpy(dic.tgt).cuda(),
                                        dic.v_src, dic.v_tgt)
    rev_full = synth.Dictionary(dic.v_tgt, dic.v_src, t_off.cpu().numpy(), t_tgt.cpu().numpy())
    rev_dic = synth.thin_dictionary(rev_full, TUNE_DICT_DROP, synth.SEED_BASE + 53)
    db = miner.DeviceBatch.from_batch(dataclasses.replace(b, dic=fwd_dic))
    plan = miner.Plan(db, options=options)
    rev = miner.Plan(db.reversed(torch.from_numpy(rev_dic.off).cuda(), torch.from_numpy(rev_dic.tgt).cuda()),
                     options=options)
    w = params.w
    prev = miner.MineParams(w=(w[1], w[0], w[2], w[3]), b=params.b, gap=params.gap, thr=params.thr)
    of, orv = plan.new_output(), rev.new_output()
    for _ in range(args.warmup):
        plan.mine(params, of)
        rev.mine(prev, orv)
        u = miner.combine_links(plan, of, rev, orv, "union")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.mine(params, of)
        rev.mine(prev, orv)
        u = miner.combine_links(plan, of, rev, orv, "union", out=u)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1000.0 / args.steps
    x = miner.combine_links(plan, of, rev, orv, "intersect")
    gold = [set(map(tuple, g.tolist())) for g in b.gold]

    def quality(links):
        tp = sum(len(l & g) for l, g in zip(links, gold))
        nl, ng = sum(len(l) for l in links), sum(len(g) for g in gold)
        p_, r_ = tp / max(nl, 1), tp / max(ng, 1)
        return {"links": nl, "correct": tp, "precision": p_, "recall": r_,
                "f1": 2 * p_ * r_ / max(p_ + r_, 1e-12)}

    def pair_sets(o, swap=False):
        off = o["link_off"].cpu().numpy()
        li, lj = o["link_i"].cpu().numpy(), o["link_j"].cpu().numpy()
        return [set(zip(lj[off[k]:off[k + 1]].tolist(), li[off[k]:off[k + 1]].tolist())) if swap else
                set(zip(li[off[k]:off[k + 1]].tolist(), lj[off[k]:off[k + 1]].tolist())) for k in range(b.n_pairs)]
    rec = {"metric": "DP cell-updates/s (bi-directional mining: both directions + union)",
           "value": 2 * plan.n_cells / secs, "ms_per_step": secs * 1e3, "pairs": b.n_pairs,
           "forward": quality(pair_sets(of)), "reverse": quality(pair_sets(orv, swap=True)),
           "union": quality(pair_sets(u)), "intersection": quality(pair_sets(x)),
           "dictionaries": f"forward and reverse each keep an independent {100 * (1 - TUNE_DICT_DROP):.0f} % of "
                           "the planting dictionary's entries",
           "reverse_classifier": "mirrored (w1, w0, w2, w3), same b, gap, thr"}
    rev.close()
    plan.close()
    return rec


def run_anchors(args):
    """Anchor tokens (Section 5.3) on planted Wikipedia-shaped pairs: the GPU
    time of extending the corpora and the dictionary, and the default
    classifier's links against the gold links without and with anchors."""
    import torch
    from paper_1512_01641_gb300 import miner
    v_anchor = 100_000
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 60))
    dic = synth.make_dictionary(rng, 50_000, 50_000)
    b = synth.tune_batch(args.anchor_pairs, seed=synth.SEED_BASE + 61, dic=dic)
    sa, ta = synth.make_anchors(b, synth.SEED_BASE + 62, v_anchor=v_anchor)
    db = miner.DeviceBatch.from_batch(b)
    dev = [(torch.from_numpy(a.sent_off).cuda(), torch.from_numpy(a.ids).cuda()) for a in (sa, ta)]
    miner.add_anchors(db, *dev, v_anchor)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ext = miner.add_anchors(db, *dev, v_anchor)
    torch.cuda.synchronize()
    extend_ms = (time.perf_counter() - t0) * 1e3

    def evaluate(batch):
        with miner.Plan(batch) as plan:
            out = plan.mine(miner.MineParams())
            gold = torch.from_numpy(miner.gold_cells(b, plan)).cuda()
            tp, nl, ng = (int(x) for x in plan.link_gold_counts(out, gold).cpu().tolist())
        p, r = tp / max(nl, 1), tp / max(ng, 1)
        return {"precision": p, "recall": r, "f1": 2 * p * r / (p + r) if p + r else 0.0, "links": nl, "gold": ng}
    return {"pairs": b.n_pairs, "v_anchor": v_anchor, "anchor_tokens": int(len(sa.ids) + len(ta.ids)),
            "extend_ms": extend_ms, "words": evaluate(db), "with_anchors": evaluate(ext)}


def _pinned_inputs(batch):
    import torch
    host = [batch.src.doc_sent_off, batch.src.sent_tok_off, batch.src.tok, batch.tgt.doc_sent_off,
            batch.tgt.sent_tok_off, batch.tgt.tok, batch.dic.off, batch.dic.tgt]
    return [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in host]


def e2e_host_abi(batch, params, steps, options=None):
    """The C ABI from host buffers: one mine_pairs_host call per step (upload
    from pinned host memory, plan, mine, download of links and scores, all
    inside the call).  Median seconds per step, bytes each way."""
    import torch
    from paper_1512_01641_gb300 import miner
    pinned = _pinned_inputs(batch)
    h2d = sum(t.numel() * t.element_size() for t in pinned)
    ns, mt = np.diff(batch.src.doc_sent_off), np.diff(batch.tgt.doc_sent_off)
    cap = max(int(np.minimum(ns, mt).sum()), 1)
    out = {"link_off": torch.empty(batch.n_pairs + 1, dtype=torch.int64).pin_memory(),
           "link_i": torch.empty(cap, dtype=torch.int32).pin_memory(),
           "link_j": torch.empty(cap, dtype=torch.int32).pin_memory(),
           "link_s": torch.empty(cap, dtype=torch.float32).pin_memory(),
           "pair_score": torch.empty(max(batch.n_pairs, 1), dtype=torch.float32).pin_memory()}
    miner.mine_host(pinned, batch.dic.v_src, batch.dic.v_tgt, params, options, out)  # warm-up
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        miner.mine_host(pinned, batch.dic.v_src, batch.dic.v_tgt, params, options, out)
        times.append(time.perf_counter() - t0)
    n = int(out["link_off"][-1])
    d2h = out["link_off"].numel() * 8 + batch.n_pairs * 4 + n * 12
    # the same uploads alone (torch copies of the eight pinned arrays, one
    # stream): what the host link gives on this machine, beside the call's time
    dev = [torch.empty_like(t, device="cuda") for t in pinned]
    copy_ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for d, t in zip(dev, pinned):
            d.copy_(t, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        copy_ms.append(e0.elapsed_time(e1))
    del dev
    return float(np.median(times)), h2d, d2h, float(np.median(copy_ms))


def e2e_pipelined(batch, params, steps, options=None):
    """Public API from pinned host buffers, batches streamed through
    BatchPipeline (the next batch's upload and plan overlap the current
    batch's mining, the previous batch's download overlaps the next mining);
    every step uploads its inputs and downloads its links.
    Seconds per step over the whole stream (pipeline fill and drain
    included)."""
    import torch
    from paper_1512_01641_gb300.pipeline import BatchPipeline
    pinned = _pinned_inputs(batch)
    pipe = BatchPipeline(params, batch.dic.v_src, batch.dic.v_tgt, options=options)
    pipe.submit(pinned)  # warm-up batch
    pipe.flush()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    got = 0
    for _ in range(steps):
        got += pipe.submit(pinned) is not None
    last = pipe.flush()
    got += last is not None
    torch.cuda.synchronize()
    secs = (time.perf_counter() - t0) / steps
    assert got == steps
    d2h = 8 + sum(t.numel() * t.element_size() for t in last.values())
    return secs, d2h


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.soft_step:
        soft_step(args)
        return
    import torch
    rank, world, lrank = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(lrank)
    from paper_1512_01641_gb300 import miner
    miner.lib(build_if_missing=True)

    batch, desc = workload(args, rank)
    params = miner.MineParams()
    db = miner.DeviceBatch.from_batch(batch)
    plan = miner.Plan(db)
    out = plan.new_output()
    tuned = None
    if not args.no_autotune:
        from paper_1512_01641_gb300 import autotune
        tuned = autotune.autotune(plan, batch, params, cache_path=None)
        tuned = {"best": tuned["best"], "fill_ms": tuned["fill_ms"], "candidates": len(tuned["trials"])}
    for _ in range(args.warmup):
        plan.mine(params, out)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(lrank) as clk:
        # timed region: K graph launches of the whole batch
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            plan.mine(params, out)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        secs = ev0.elapsed_time(ev1) / 1000.0
        # per-kernel pass: the same K steps launched directly, each kernel
        # bracketed by CUDA events on its launching stream
        plan.set_timing(True)
        ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev2.record(stream)
        for _ in range(args.steps):
            plan.mine(params, out)
        ev3.record(stream)
        torch.cuda.synchronize()
        secs_direct = ev2.elapsed_time(ev3) / 1000.0
        kt = plan.kernel_times()
        plan.set_timing(False)
    clocks = clk.summary()
    plan.check()
    if world > 1:
        t = torch.tensor([secs], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        secs = float(t.item())
    cells_step = plan.n_cells * world
    value = cells_step * args.steps / secs
    pairs_s = plan.n_pairs * world * args.steps / secs
    launches = sum(n for _, n in kt.values())

    # roofline of the dominant kernel: ALU issue bound (integer compares,
    # hashing and bit-sliced counting for the counts; FP adds and selects for
    # the DP -- no dense contraction anywhere)
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / max(kt[dom][1], 1)
    n_cells = plan.n_cells
    if dom == "count":
        ops = merge_compare_ops(batch)
    else:
        ops = (OPS_SIM + OPS_DP) * n_cells
    achieved = ops / (dom_ms / 1000.0) / 1e12
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    n_sms = sm_count()
    peak = n_sms * LANES_PER_SM * sm_max * 1e6 / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": traffic_per_launch(dom, n_cells),
                "ops_per_launch": ops, "ms_per_launch": dom_ms,
                "peak_basis": f"model, not a measurement: {n_sms} SMs (read from the device) x {LANES_PER_SM} "
                              f"lane-ops/clk (one warp instruction per sub-partition per clock) x {sm_max:.0f} MHz"}
    n_links = int(out["link_off"][-1].item())
    hbm_gbs, hbm_src = hbm_peak()
    alg = algorithmic_bytes(batch, n_links)
    hbm = {"algorithmic_bytes_per_step": alg, "achieved_gbs": alg / (secs / args.steps) / 1e9, "peak_gbs": hbm_gbs,
           "peak_source": hbm_src, "frac": alg / (secs / args.steps) / 1e9 / hbm_gbs,
           "count_kernel_dram_bytes_per_launch": traffic_per_launch("count", n_cells)}

    # NW only: fill, walk, link scoring and compaction from the batch's cached counts
    nw_only = None
    if not args.no_configs:
        counts = plan.count()
        out_nw = plan.new_output()
        t_nw = timed_steps(lambda: plan.align(params, counts, out_nw), args.steps, 1)
        nw_only = {"value": n_cells * args.steps / t_nw, "unit": UNIT, "ms_per_step": 1000 * t_nw / args.steps,
                   "what": "mine_align from cached counts (fill, traceback, link scoring, compaction)"}
        del counts, out_nw

    anchors_rec = None
    if rank == 0 and not args.no_anchors:
        anchors_rec = run_anchors(args)

    bi_rec = None
    if not args.no_bi:
        bi_rec = run_bi(args, params, {})  # its own 10,000-pair batch: the plan defaults

    e2e = None
    if not args.no_e2e:
        plan_keep = plan
        opts = dict(tuned["best"]) if tuned else {}
        e_abi, h2d, d2h, copy_ms = e2e_host_abi(batch, params, args.e2e_steps, opts)
        e_t, d2h_p = e2e_pipelined(batch, params, args.e2e_stream_steps, opts)
        e2e = {"value": cells_step / world / e_abi * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "seconds_per_step": e_abi,
               "includes": "one mine_pairs_host C-ABI call per step: H2D of the inputs from pinned host memory, "
                           "plan creation (validation, geometry, scratch), mining, D2H of links and scores "
                           f"(median of {args.e2e_steps} steps)",
               "plan_options": opts,
               "h2d_copy_alone": {"ms": copy_ms, "gbs": h2d / copy_ms / 1e6,
                                  "what": "the eight input arrays copied alone from pinned host memory "
                                          "(torch copies, one stream, median of 3)"},
               "pipelined": {"value": cells_step / world / e_t * world, "seconds_per_step": e_t,
                             "d2h_bytes_per_step": d2h_p,
                             "includes": "the same work streamed batch after batch through BatchPipeline (the "
                                         "next batch's upload and plan overlap the current mining; "
                                         f"{args.e2e_stream_steps} steps incl. pipeline fill and drain)"}}
        plan = plan_keep

    cpu = ties = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, pick, ref = cpu_baseline(batch, args.cpu_pairs)
        out_all = plan.mine(miner.MineParams(thr=-1.0))
        ties = near_tie_record(batch, out_all, pick, ref, params.gap)
        del out_all

    configs = None
    if rank == 0 and not args.no_configs:
        configs = config_records(args, params)

    tune_rec = None
    if rank == 0 and not args.no_tune:
        try:
            tune_rec = run_tune(args)
        except Exception as exc:  # the tuning comparison must not lose the bench line
            tune_rec = {"error": f"{type(exc).__name__}: {exc}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded, Wikipedia-shaped)", "config": desc,
                "pairs_per_s": pairs_s, "gpu_launches": launches,
                "kernel_ms": {k: v[0] / max(args.steps, 1) for k, v in kt.items() if v[1]},
                "direct_launch_ms_per_step": 1000 * secs_direct / args.steps,
                "graph": {"captures": plan.get_option("graph_captures")},
                "autotune": tuned, "tune": tune_rec, "bi": bi_rec, "anchors": anchors_rec,
                "roofline": roofline, "hbm": hbm, "nw_only": nw_only, "near_ties": ties, "configs": configs,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "sm_count": sm_count()}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
