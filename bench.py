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
N_SMS = 152
LANES_PER_SM = 128  # 4 sub-partitions x 32 lanes issue per clock
# algorithmic lane-operations per cell of the roofline model when the path is
# timed from precomputed counts (similarity and DP only)
OPS_SIM = 11   # 4 quotients, 4 multiply-adds, exp, add, reciprocal
OPS_DP = 8     # 3 candidates, 2 max, 2 compare/select, 1 pack


# DRAM bytes per cell of the dominant kernels, from one ncu capture
# (profiles/), valid only while the kernel's source is unchanged.
TRAFFIC = {
    "count": {"file": "paper_1512_01641_gb300/csrc/count.cu", "sha1": "fc41409cb6928eee2ef0d627715880e23eb71df0",
              "bytes_per_cell": (264.148992e6 + 409.225216e6) / 218470577},
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
    ap.add_argument("--anchor-pairs", type=int, default=10_000)
    ap.add_argument("--soft-step", action="store_true",
                    help="only time one soft-NW forward+backward on a 4,096-pair tuning minibatch (profiling)")
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
                      f"{dt:.1f} s", "seconds": dt, "cells": cells}


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
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 40))
    dic = synth.make_dictionary(rng, 50_000, 50_000)
    td = tune.TuneData(synth.tune_batch(4096, seed=synth.SEED_BASE + 4, dic=dic))
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
    print(json.dumps({"soft_step": {"pairs": td.plan.n_pairs, "cells": td.plan.n_cells, "gamma": 0.1,
                                    "forward_ms": ev[0].elapsed_time(ev[1]),
                                    "backward_ms": ev[1].elapsed_time(ev[2])}}))


def run_tune(args):
    """Soft-NW gradient tuning (Adam) vs the 7^3 grid search and the paper's
    random search (343 draws), same GPU, evaluated by hard-NW micro-F1 on
    held-out planted pairs."""
    from paper_1512_01641_gb300 import tune
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 40))
    dic = synth.make_dictionary(rng, 50_000, 50_000)
    tr = synth.tune_batch(args.tune_pairs, seed=synth.SEED_BASE + 4, dic=dic)
    ev = synth.tune_batch(args.tune_eval, seed=synth.SEED_BASE + 5, dic=dic)
    r = tune.compare(tr, ev, steps=args.tune_steps)
    r["train_cells"] = tr.cells()
    return r


def run_bi(args, db, plan, params, options):
    """Bi-directional mining (Section 5.4, BI) of the same batch: the reverse
    direction by a plan over the reversed batch (dictionary transposed on the
    GPU), mined with the mirrored classifier (the two overlap weights
    exchanged), then the per-pair union of the links.  Device-timed like the
    main line: K steps of forward mining + reverse mining + combination."""
    import torch
    from paper_1512_01641_gb300 import miner
    rev = miner.Plan(db.reversed(), options=options)
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
    rec = {"metric": "DP cell-updates/s (bi-directional mining: both directions + union)",
           "value": 2 * plan.n_cells / secs, "ms_per_step": secs * 1e3,
           "links_fwd": int(of["link_off"][-1]), "links_rev": int(orv["link_off"][-1]),
           "links_union": int(u["link_off"][-1]), "links_intersect": int(x["link_off"][-1]),
           "reverse_classifier": "mirrored (w1, w0, w2, w3), same b, gap, thr; transposed dictionary"}
    rev.close()
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


def e2e_run(batch, params, steps, options=None):
    """Public API from pinned host buffers, one batch at a time: upload,
    plan (with the given plan options), mine, download, destroy.  Median
    seconds per step."""
    import torch
    from paper_1512_01641_gb300 import miner
    pinned = _pinned_inputs(batch)
    h2d = sum(t.numel() * t.element_size() for t in pinned)
    times, d2h = [], 0
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dev = [t.to("cuda", non_blocking=True) for t in pinned]
        db = miner.DeviceBatch(*dev, batch.dic.v_src, batch.dic.v_tgt)
        plan = miner.Plan(db, options=options)
        out = plan.mine(params)
        n = int(out["link_off"][-1].item())
        res = {"link_off": out["link_off"].cpu(), "pair_score": out["pair_score"].cpu(),
               "link_i": out["link_i"][:n].cpu(), "link_j": out["link_j"][:n].cpu(), "link_s": out["link_s"][:n].cpu()}
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        d2h = 8 + sum(t.numel() * t.element_size() for t in res.values())
        plan.close()
        del dev, db, out
    return float(np.median(times)), h2d, d2h


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
    peak = N_SMS * LANES_PER_SM * sm_max * 1e6 / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": traffic_per_launch(dom, n_cells),
                "ops_per_launch": ops, "ms_per_launch": dom_ms,
                "peak_basis": f"{N_SMS} SMs x {LANES_PER_SM} lane-ops/clk x {sm_max:.0f} MHz (max SM clock)"}

    anchors_rec = None
    if rank == 0 and not args.no_anchors:
        anchors_rec = run_anchors(args)

    bi_rec = None
    if not args.no_bi:
        bi_rec = run_bi(args, db, plan, params, dict(tuned["best"]) if tuned else {})

    e2e = None
    if not args.no_e2e:
        plan_keep = plan
        opts = dict(tuned["best"]) if tuned else {}
        e_seq, h2d, d2h = e2e_run(batch, params, args.e2e_steps, opts)
        e_t, d2h_p = e2e_pipelined(batch, params, args.e2e_stream_steps, opts)
        e2e = {"value": cells_step / world / e_t * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h_p, "seconds_per_step": e_t,
               "includes": "per step: H2D of the inputs from pinned host memory, plan creation (validation, "
                           "geometry, scratch), mine_pairs, D2H of links and scores; batches streamed "
                           f"through BatchPipeline ({args.e2e_stream_steps} steps incl. pipeline fill and drain)",
               "plan_options": opts,
               "sequential": {"value": cells_step / world / e_seq * world, "seconds_per_step": e_seq,
                              "includes": "one batch at a time, nothing overlapped"}}
        plan = plan_keep

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(batch, args.cpu_pairs)

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
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
