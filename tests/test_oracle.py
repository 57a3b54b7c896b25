"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here touches the CUDA path: the oracle is checked against the paper's
worked examples (Figures 4 and 6), hand-worked Eq. (1) tables, closed forms,
invariants and brute-force enumeration of every monotone alignment.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1512_01641_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _identity_sim(rows, cols):
    return np.array([[1.0 if r == c else 0.0 for c in cols] for r in rows])


def _path_cells(moves, N, M):
    """0-based cells visited by the path (the X marks of Figures 3-4)."""
    i = j = 0
    cells = []
    for m in moves[::-1]:
        if m == oracle.MOVE_DIAG:
            i, j = i + 1, j + 1
        elif m == oracle.MOVE_UP:
            i += 1
        else:
            j += 1
        cells.append((i - 1 if i else 0, j - 1 if j else 0))
    return cells


# ---------------------------------------------------------------- Section 5.1
def test_figure4_path_and_tie_rule():
    g = _load("fig4_nw.json")
    s = _identity_sim(g["rows"], g["cols"])
    H, mv, diag = oracle.nw(s, g["gap"])
    assert H[-1, -1] == g["score"]
    assert diag == [tuple(x) for x in g["diag"]]
    assert _path_cells(mv, 5, 5) == [tuple(x) for x in g["path_cells"]]
    # the printed two-line alignment
    cols, rows = [], []
    i = j = 0
    for m in mv[::-1]:
        if m == oracle.MOVE_DIAG:
            cols.append(g["cols"][j]); rows.append(g["rows"][i]); i += 1; j += 1
        elif m == oracle.MOVE_UP:
            cols.append("-"); rows.append(g["rows"][i]); i += 1
        else:
            cols.append(g["cols"][j]); rows.append("-"); j += 1
    assert cols == g["alignment_cols"] and rows == g["alignment_rows"]
    # brute force: two optimal alignments exist; the figure shows the one the
    # UP-first tie rule picks
    best, arg = brute.hard(s.tolist(), g["gap"])
    assert best == g["score"] and len(arg) == g["n_optimal_alignments"]
    assert tuple(map(tuple, g["diag"])) in arg


def test_figure6_unique_optimum():
    g = _load("fig6_nw.json")
    s = _identity_sim(g["rows"], g["cols"])
    H, mv, diag = oracle.nw(s, g["gap"])
    assert H[-1, -1] == g["score"]
    assert diag == [tuple(x) for x in g["diag"]]
    best, arg = brute.hard(s.tolist(), g["gap"])
    assert best == g["score"] and len(arg) == 1 and list(arg[0]) == diag


@pytest.mark.parametrize("case", range(3))
def test_eq1_hand_worked(case):
    c = _load("eq1_hand.json")["cases"][case]
    s = np.array([[1.0 if a == b else -1.0 for b in c["cols"]] for a in c["rows"]])
    H, mv, diag = oracle.nw(s, c["gap"])
    assert np.array_equal(H, np.array(c["H"], float))
    assert H[-1, -1] == c["score"]
    assert diag == [tuple(x) for x in c["diag"]]


def test_gap_tie_prefers_up():
    # H(1,1) = max(-5, -2, -2): UP and LEFT tie; the oracle walks UP first.
    H, mv, diag = oracle.nw(np.array([[-5.0]]), 1.0)
    assert H[1, 1] == -2.0 and list(mv) == [oracle.MOVE_UP, oracle.MOVE_LEFT] and diag == []


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_hard(seed):
    rng = np.random.default_rng(seed)
    N, M = rng.integers(1, 7, size=2)
    if seed % 2:  # a small value set makes exact ties common
        s = rng.choice([0.0, 0.25, 0.5, 0.75, 1.0], size=(N, M))
        p = 0.125
    else:
        s = rng.random((N, M))
        p = float(rng.choice([0.05, 0.3, 0.6]))
    H, mv, diag = oracle.nw(s, p)
    best, arg = brute.hard(s.tolist(), p)
    assert abs(H[-1, -1] - best) < 1e-12
    assert tuple(diag) in arg
    assert abs(oracle.path_score(s, p, diag) - best) < 1e-12


def test_empty_sides():
    for N, M in [(0, 0), (0, 4), (3, 0)]:
        H, mv, diag = oracle.nw(np.zeros((N, M)), 0.3)
        assert H[-1, -1] == pytest.approx(-0.3 * (N + M)) and diag == []
        assert len(mv) == N + M


@pytest.mark.parametrize("N,M,c,p", [(5, 9, 0.7, 0.3), (12, 4, 0.2, 0.1), (7, 7, -0.1, 0.3), (1, 6, 0.9, 0.5)])
def test_constant_similarity_closed_form(N, M, c, p):
    # with c + 2p > 0 a diagonal step beats an UP+LEFT detour, so the optimum
    # takes min(N,M) diagonals and |N-M| gaps
    H, _, diag = oracle.nw(np.full((N, M), c), p)
    assert H[-1, -1] == pytest.approx(min(N, M) * c - p * abs(N - M), abs=1e-12)
    assert len(diag) == min(N, M)


def test_single_row_closed_form():
    rng = np.random.default_rng(7)
    for _ in range(20):
        M = int(rng.integers(1, 12))
        s = rng.random((1, M)) * 2 - 1
        p = float(rng.random())
        expect = max(s.max() - p * (M - 1), -p * (M + 1))
        H, _, _ = oracle.nw(s, p)
        assert H[-1, -1] == pytest.approx(expect, abs=1e-12)
        H2, _, _ = oracle.nw(s.T.copy(), p)
        assert H2[-1, -1] == pytest.approx(expect, abs=1e-12)


# ---------------------------------------------------------------- features
def _dic(lists, v_tgt=100):
    off = np.zeros(len(lists) + 1, np.int32)
    off[1:] = np.cumsum([len(l) for l in lists])
    return synth.Dictionary(len(lists), v_tgt, off, np.asarray([t for l in lists for t in sorted(l)], np.int32))


def test_counts_hand_worked():
    # source ids 0..4; 0->{10,11}, 1->{12}, 2->{13,14,15}, 3->{10}, 4->{16}
    dic = _dic([[10, 11], [12], [13, 14, 15], [10], [16]])
    # src [0,0,1,3]: positions 0,1 (id 0: 10/11), 2 (id 1: 12), 3 (id 3: 10)
    # tgt [10,10,12,20]: 10 hits positions 0,1,3; 12 hits position 2
    assert oracle.counts([0, 0, 1, 3], [10, 10, 12, 20], dic) == (4, 3)
    # tgt [11,13]: 11 via id 0 (positions 0,1); 13 not a translation of src
    assert oracle.counts([0, 0, 1, 3], [11, 13], dic) == (2, 1)
    assert oracle.counts([2, 4], [13, 15, 16, 16], dic) == (2, 4)
    assert oracle.counts([1], [10, 11], dic) == (0, 0)


def test_counts_invariants_and_swap_symmetry():
    rng = np.random.default_rng(3)
    v_src, v_tgt = 30, 25
    lists = [sorted(set(rng.integers(0, v_tgt, size=int(rng.integers(1, 4))).tolist())) for _ in range(v_src)]
    dic = _dic(lists, v_tgt)
    # inverse dictionary: target id -> source ids translating to it
    inv = [[] for _ in range(v_tgt)]
    for s_id, l in enumerate(lists):
        for t in l:
            inv[t].append(s_id)
    inv = [l if l else [] for l in inv]
    dinv = _dic(inv, v_src)
    for _ in range(300):
        src = sorted(rng.integers(0, v_src, size=int(rng.integers(1, 12))).tolist())
        tgt = sorted(rng.integers(0, v_tgt, size=int(rng.integers(1, 12))).tolist())
        ms, mt = oracle.counts(src, tgt, dic)
        assert 0 <= ms <= len(src) and 0 <= mt <= len(tgt)
        # t is a translation of s iff s is an inverse translation of t, so the
        # roles of ms and mt swap
        ms2, mt2 = oracle.counts(tgt, src, dinv)
        assert (ms2, mt2) == (mt, ms)


def test_counts_full_translation():
    # a target built by translating every source position hits every position
    rng = np.random.default_rng(5)
    b = synth.make_batch(11, 4, v_src=500, v_tgt=500)
    for _ in range(100):
        src = np.sort(rng.integers(0, 500, size=int(rng.integers(5, 31)))).astype(np.int32)
        tgt = np.sort([rng.choice(b.dic.translations(v)) for v in src]).astype(np.int32)
        assert oracle.counts(src, tgt, b.dic) == (len(src), len(tgt))


def test_counts_multiplicity():
    dic = _dic([[5], [6]])
    # repeated source tokens count once per position; repeated targets too
    assert oracle.counts([0, 0, 0, 1], [5, 5], dic) == (3, 2)
    assert oracle.counts([0], [5, 5, 5, 7], dic) == (1, 3)


def test_float32_ratio_equals_rounded_double():
    # the CUDA path divides in FP32 with IEEE rounding; the oracle rounds the
    # FP64 quotient.  For every ratio that can occur (counts <= length <= 64)
    # the two agree bit for bit.
    a = np.arange(65)
    A, B = np.meshgrid(a, a[1:], indexing="ij")
    q32 = A.astype(np.float32) / B.astype(np.float32)
    q64 = (A.astype(np.float64) / B.astype(np.float64)).astype(np.float32)
    assert np.array_equal(q32.view(np.uint32), q64.view(np.uint32))


def test_features_and_similarity():
    f = oracle.features(3, 2, 6, 4)
    assert np.allclose(f, [0.5, 0.5, 2 / 6, 4 / 6], rtol=0, atol=1e-15)
    w = [4.0, 4.0, -2.0, 1.0]
    z = 4 * 0.5 + 4 * 0.5 - 2 * (2 / 6) + (4 / 6) - 3.0
    assert oracle.similarity(f, w, -3.0) == pytest.approx(1 / (1 + math.exp(-z)), rel=1e-15)
    # |ls-lt|/max + min/max == 1 always
    for ls in range(1, 40):
        for lt in range(1, 40):
            g = oracle.features(0, 0, ls, lt)
            assert g[2] + g[3] == pytest.approx(1.0, abs=1e-15)


def test_mine_links_are_thresholded_path():
    b = synth.single_pair()
    w = [4.0, 4.0, -2.0, 1.0]
    r = oracle.mine(b, w, -3.0, 0.3, 0.5, want_counts=True)
    ms, mt = r["counts"][0][..., 0], r["counts"][0][..., 1]
    src, tgt = b.src.doc(0), b.tgt.doc(0)
    # counts from the batch driver equal the single-pair routine
    for i in range(0, 40, 7):
        for j in range(0, 45, 5):
            assert (ms[i, j], mt[i, j]) == oracle.counts(src[i], tgt[j], b.dic)
    S = np.array([[oracle.similarity(oracle.features(ms[i, j], mt[i, j], len(src[i]), len(tgt[j])), w, -3.0)
                   for j in range(45)] for i in range(40)])
    H, _, diag = oracle.nw(S, 0.3)
    assert r["score"][0] == H[-1, -1]
    assert [(i, j) for i, j, _ in r["diag"][0]] == diag
    assert all(s >= 0.5 for _, _, s in r["links"][0])
    assert [x for x in r["diag"][0] if x[2] >= 0.5] == r["links"][0]


# ---------------------------------------------------------------- soft NW
def test_soft_closed_form_zero_scores():
    # s = 0, p = 0: every alignment scores 0, so V = gamma ln D(N,M) and a cell
    # is taken diagonally by D(i-1,j-1) D(N-i,M-j) of the D(N,M) paths
    for N, M in [(1, 1), (3, 5), (6, 6), (8, 3)]:
        for g in [1.0, 0.1]:
            V, E, _ = oracle.soft_nw(np.zeros((N, M)), 0.0, g)
            D = brute.delannoy(N, M)
            assert V[-1, -1] == pytest.approx(g * math.log(D), rel=1e-12)
            for i in range(1, N + 1):
                for j in range(1, M + 1):
                    e = brute.delannoy(i - 1, j - 1) * brute.delannoy(N - i, M - j) / D
                    assert E[i - 1, j - 1] == pytest.approx(e, rel=1e-12)


@pytest.mark.parametrize("seed", range(12))
def test_soft_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    N, M = rng.integers(1, 6, size=2)
    s = rng.random((N, M))
    p = float(rng.choice([0.05, 0.3]))
    g = float(rng.choice([1.0, 0.1, 0.01]))
    V, E, dp = oracle.soft_nw(s, p, g)
    v, Eb = brute.soft(s.tolist(), p, g)
    assert V[-1, -1] == pytest.approx(v, rel=1e-12, abs=1e-12)
    assert np.allclose(E, np.array(Eb), rtol=1e-9, atol=1e-12)
    # dV/dp = -(expected number of gap steps) = -(N + M - 2 * expected diagonals)
    assert dp == pytest.approx(-(N + M - 2 * np.sum(Eb)), rel=1e-9, abs=1e-12)
    # hard value <= soft value <= hard value + gamma ln D
    H, _, _ = oracle.nw(s, p)
    assert H[-1, -1] - 1e-12 <= V[-1, -1] <= H[-1, -1] + g * math.log(brute.delannoy(N, M)) + 1e-12


@pytest.mark.slow
def test_soft_brute_force_8x8():
    rng = np.random.default_rng(8)
    s = rng.random((8, 8))
    V, E, _ = oracle.soft_nw(s, 0.3, 0.1)
    v, Eb = brute.soft(s.tolist(), 0.3, 0.1)
    assert V[-1, -1] == pytest.approx(v, rel=1e-12)
    assert np.allclose(E, np.array(Eb), rtol=1e-9, atol=1e-12)


def test_soft_tends_to_hard():
    rng = np.random.default_rng(9)
    s = rng.random((9, 11))
    H, _, diag = oracle.nw(s, 0.3)
    V, E, _ = oracle.soft_nw(s, 0.3, 1e-3)
    assert V[-1, -1] == pytest.approx(H[-1, -1], abs=1e-3 * math.log(brute.delannoy(9, 11)) + 1e-9)
    hard = np.zeros_like(s)
    for i, j in diag:
        hard[i, j] = 1
    assert np.abs(E - hard).max() < 1e-6


def test_soft_adjoint_equals_autograd():
    torch = pytest.importorskip("torch")
    from oracle import softgrad
    rng = np.random.default_rng(12)
    s = rng.random((6, 7))
    V, E, dp = oracle.soft_nw(s, 0.3, 0.1)
    st = torch.tensor(s, requires_grad=True)
    pt = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    v = softgrad.soft_value(st, pt, 0.1)
    gs, gp = torch.autograd.grad(v, [st, pt])
    assert float(v.detach()) == pytest.approx(V[-1, -1], rel=1e-12)
    assert np.allclose(gs.numpy(), E, rtol=1e-10, atol=1e-13)
    assert float(gp) == pytest.approx(dp, rel=1e-10)


def _soft_pairs(seed, n_pairs=3, n=8):
    b = synth.make_batch(seed, n_pairs, v_src=300, v_tgt=300, planted_frac=1.0,
                         src_sizes=np.full(n_pairs, n), p_ins=0.0, p_sdrop=0.0)
    r = oracle.mine(b, [4, 4, -2, 1], -3, 0.3, 0.5, want_counts=True)
    pairs = []
    for k in range(n_pairs):
        c = r["counts"][k]
        ls = [len(x) for x in b.src.doc(k)]
        lt = [len(x) for x in b.tgt.doc(k)]
        gold = np.zeros(c.shape[:2])
        for i, j in b.gold[k]:
            gold[i, j] = 1
        pairs.append((c[..., 0], c[..., 1], ls, lt, gold))
    return pairs


@pytest.mark.parametrize("gamma", [1.0, 0.1])
def test_soft_loss_gradient_central_differences(gamma):
    pytest.importorskip("torch")
    from oracle import softgrad
    pairs = _soft_pairs(21)
    theta = np.array([4.0, 4.0, -2.0, 1.0, -3.0, 0.3, 0.5])
    L, g = softgrad.loss_and_grad(pairs, theta, gamma, 0.05)
    h = 1e-6
    for k in range(7):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (softgrad.loss_value(pairs, tp, gamma, 0.05) - softgrad.loss_value(pairs, tm, gamma, 0.05)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-4, abs=1e-7), k


def test_soft_loss_hand_worked():
    """The oracle's loss (gate, clamp, BCE mean over cells) against a 1x1 and a
    1x2 pair worked out in closed form by path enumeration
    (tests/golden/soft_loss_hand.py holds the derivation); the oracle's soft
    value and expected alignment of the same similarities too."""
    pytest.importorskip("torch")
    from oracle import softgrad
    d = _load("soft_loss_hand.json")
    pairs = [(np.array(p["ms"]), np.array(p["mt"]), p["ls"], p["lt"], np.array(p["gold"], float)) for p in d["pairs"]]
    L = softgrad.loss_value(pairs, d["theta"], d["gamma"], d["tau"], d["eps"])
    assert L == pytest.approx(d["loss"], rel=1e-10)
    assert L != pytest.approx(d["loss"] * 3 / 2, rel=1e-3)  # a mean over pairs would differ
    for p in d["pairs"]:
        V, E, _ = oracle.soft_nw(np.array(p["s"]), d["theta"][5], d["gamma"])
        assert V[-1, -1] == pytest.approx(p["V"], rel=1e-12)
        assert np.allclose(E, np.array(p["E"]), rtol=1e-10, atol=1e-15)
    # the clamp acts on the second pair's unmatched cell
    assert d["pairs"][1]["P"][0][1] == d["eps"]


# --- the tuning objective (Section 5.2): similarity of automatic and human alignments ---

def _lcs_brute(a, b):
    """Longest common subsequence by enumerating every subsequence of a."""
    import itertools
    best = 0
    for r in range(len(a) + 1):
        for idx in itertools.combinations(range(len(a)), r):
            sub = [a[x] for x in idx]
            it = iter(b)
            if all(any(y == x for y in it) for x in sub):
                best = max(best, r)
    return best


def test_nw_similarity_hand_cases():
    from oracle import evaluate
    assert evaluate.nw_matched([(0, 0), (1, 1), (2, 2)], [(0, 0), (2, 2)]) == 2
    assert evaluate.nw_matched([], [(0, 0)]) == 0
    # order matters (an alignment of sequences, not a set overlap)
    assert evaluate.nw_matched([(0, 0), (1, 1)], [(1, 1), (0, 0)]) == 1
    r = evaluate.similarity([[(0, 0), (1, 1), (2, 2)]], [[(0, 0), (2, 2)]])
    assert (r["matched"], r["auto"], r["human"]) == (2, 3, 2)
    assert r["similarity"] == pytest.approx(0.8)


@pytest.mark.parametrize("seed", range(6))
def test_nw_similarity_equals_lcs_brute_force(seed):
    from oracle import evaluate
    rng = np.random.default_rng(seed)
    for _ in range(20):
        a = [tuple(x) for x in rng.integers(0, 3, size=(int(rng.integers(0, 7)), 2))]
        b = [tuple(x) for x in rng.integers(0, 3, size=(int(rng.integers(0, 7)), 2))]
        assert evaluate.nw_matched(a, b) == _lcs_brute(a, b)


@pytest.mark.parametrize("seed", range(4))
def test_nw_similarity_of_monotone_alignments_is_their_intersection(seed):
    # two link lists taken from monotone paths: the NW alignment pairs up
    # exactly the common links, so the similarity is the links' micro-F1
    from oracle import evaluate
    rng = np.random.default_rng(100 + seed)
    for _ in range(30):
        n, m = int(rng.integers(1, 40)), int(rng.integers(1, 40))

        def monotone():
            k = int(rng.integers(0, min(n, m) + 1))
            i = np.sort(rng.choice(n, k, replace=False))
            j = np.sort(rng.choice(m, k, replace=False))
            return [(int(x), int(y)) for x, y in zip(i, j)]
        a, b = monotone(), monotone()
        assert evaluate.nw_matched(a, b) == len(set(a) & set(b))


# --- bi-directional mining (Section 5.4, BI) ---

def _random_dict(seed, v_src=60, v_tgt=40, kmax=4):
    rng = np.random.default_rng(seed)
    lists = [sorted(rng.choice(v_tgt, int(rng.integers(0, kmax + 1)), replace=False).tolist()) for _ in range(v_src)]
    off = np.zeros(v_src + 1, np.int32)
    off[1:] = np.cumsum([len(x) for x in lists])
    return synth.Dictionary(v_src, v_tgt, off, np.array([t for x in lists for t in x], np.int32))


@pytest.mark.parametrize("seed", range(3))
def test_dictionary_transpose_is_the_inverse_relation(seed):
    from oracle import bi
    d = _random_dict(seed)
    r = bi.transpose_dictionary(d)
    assert (r.v_src, r.v_tgt) == (d.v_tgt, d.v_src) and len(r.tgt) == len(d.tgt)
    for t in range(d.v_tgt):
        lst = r.tgt[r.off[t]:r.off[t + 1]].tolist()
        assert lst == sorted(set(lst))
        assert set(lst) == {v for v in range(d.v_src) if t in d.tgt[d.off[v]:d.off[v + 1]]}
    rr = bi.transpose_dictionary(r)
    assert np.array_equal(rr.off, d.off) and np.array_equal(rr.tgt, d.tgt)


@pytest.mark.parametrize("seed", range(3))
def test_reverse_counts_with_the_transposed_dictionary_are_swapped(seed):
    # ms of the reverse direction counts target positions whose token has a
    # (reverse) translation in the source sentence: that is the forward mt,
    # and the reverse mt is the forward ms
    from oracle import bi
    rng = np.random.default_rng(10 + seed)
    d = _random_dict(20 + seed)
    r = bi.transpose_dictionary(d)
    for _ in range(50):
        src = np.sort(rng.integers(0, d.v_src, int(rng.integers(1, 12))))
        tgt = np.sort(rng.integers(0, d.v_tgt, int(rng.integers(1, 12))))
        ms, mt = oracle.counts(src, tgt, d)
        assert oracle.counts(tgt, src, r) == (mt, ms)


def test_reverse_mining_of_the_transposed_problem_has_the_same_optimum():
    # with the transposed dictionary and the two overlap weights exchanged the
    # reverse similarity matrix is the transpose of the forward one, so every
    # pair's optimum H(N, M) is unchanged
    from oracle import bi
    b = synth.make_batch(71, 6, v_src=3000, v_tgt=3000, size_median=20, size_hi=40)
    w, bias, gap, thr = np.array([4.0, 3.0, -2.0, 1.0]), -3.0, 0.3, 0.5
    f = oracle.mine(b, w, bias, gap, thr)
    r = oracle.mine(bi.reversed_batch(b), w[[1, 0, 2, 3]], bias, gap, thr)
    assert np.allclose(f["score"], r["score"], rtol=0, atol=1e-12)


def test_combine_links_hand_case():
    from oracle import bi
    fwd = [[(0, 0, 0.9), (2, 1, 0.8)]]
    rev = [[(1, 2, 0.7), (3, 3, 0.6)]]  # reverse coordinates: (j, i)
    u = bi.combine(fwd, rev, "union")[0]
    assert [(i, j) for i, j, _, _ in u] == [(0, 0), (2, 1), (3, 3)]
    assert u[1][2:] == (0.8, 0.7)
    assert math.isnan(u[0][3]) and math.isnan(u[2][2])
    x = bi.combine(fwd, rev, "intersect")[0]
    assert [(i, j) for i, j, _, _ in x] == [(2, 1)]


# --- anchors (Section 5.3): shared names, dates, numbers, references ---

@pytest.mark.parametrize("seed", range(3))
def test_anchor_extension_adds_shared_anchor_positions_to_the_counts(seed):
    # closed form: with anchors as self-translating tokens, ms gains the
    # source anchor positions whose anchor the target sentence carries and mt
    # the target anchor positions whose anchor the source sentence carries;
    # nothing else changes (anchor ids never meet word ids)
    from oracle import anchors
    b = synth.make_batch(300 + seed, 6, v_src=2000, v_tgt=2000, planted_frac=0.5, size_median=12, size_hi=30)
    sa, ta = synth.make_anchors(b, 400 + seed, v_anchor=40, p_anchor=0.7)
    e = anchors.extend_batch(b, sa, ta, 40)
    rng = np.random.default_rng(seed)
    n_s, n_t = len(b.src.sent_tok_off) - 1, len(b.tgt.sent_tok_off) - 1
    for _ in range(200):
        i, j = int(rng.integers(n_s)), int(rng.integers(n_t))
        ms, mt = oracle.counts(b.src.sentence(i), b.tgt.sentence(j), b.dic)
        xs, xt = anchors.shared_positions(sa.ids[sa.sent_off[i]:sa.sent_off[i + 1]],
                                          ta.ids[ta.sent_off[j]:ta.sent_off[j + 1]])
        assert oracle.counts(e.src.sentence(i), e.tgt.sentence(j), e.dic) == (ms + xs, mt + xt)
        assert len(e.src.sentence(i)) == len(b.src.sentence(i)) + sa.sent_off[i + 1] - sa.sent_off[i]


def test_anchor_dictionary_entries_are_identities():
    from oracle import anchors
    d = _random_dict(7)
    e = anchors.extend_dictionary(d, 5)
    assert (e.v_src, e.v_tgt) == (d.v_src + 5, d.v_tgt + 5)
    assert np.array_equal(e.off[:d.v_src + 1], d.off) and np.array_equal(e.tgt[:len(d.tgt)], d.tgt)
    for a in range(5):
        assert e.tgt[e.off[d.v_src + a]:e.off[d.v_src + a + 1]].tolist() == [d.v_tgt + a]


def test_planted_anchors_follow_the_gold_links():
    b = synth.make_batch(310, 8, planted_frac=1.0, size_median=15, size_hi=40)
    sa, ta = synth.make_anchors(b, 311, p_keep=1.0)
    for k, g in enumerate(b.gold):
        s0, t0 = b.src.doc_sent_off[k], b.tgt.doc_sent_off[k]
        for i, j in g.tolist():
            assert (ta.ids[ta.sent_off[t0 + j]:ta.sent_off[t0 + j + 1]].tolist() ==
                    sa.ids[sa.sent_off[s0 + i]:sa.sent_off[s0 + i + 1]].tolist())


# --- the unconstrained (Yalign A*) aligner of Section 5.1, Figures 3 and 5 ---

def _score_choice(s, p, choice):
    """Score of a row-by-row choice, written out for the brute force: a match
    ahead of the pointer skips the columns between (p each), a match at or
    behind it is a move back (p), an unmatched row costs p, and so does every
    target sentence after the final pointer."""
    N, M = s.shape
    ptr, tot = 0, 0.0
    for i in range(N):
        j = choice[i]
        if j is None:
            tot -= p
        elif j + 1 > ptr:
            tot += s[i, j] - p * (j - ptr)
            ptr = j + 1
        else:
            tot += s[i, j] - p
            ptr = j + 1
    return tot - p * (M - ptr)


@pytest.mark.parametrize("name", ["fig3_unconstrained.json", "fig5_unconstrained.json"])
def test_unconstrained_figures(name):
    from oracle import unconstrained
    g = _load(name)
    s = _identity_sim(g["rows"], g["cols"])
    score, links = unconstrained.align(s, g["gap"])
    assert score == g["score"]
    assert [list(x) for x in links] == g["links"]
    if "alignment_cols" in g:  # the alignment printed under Figure 3
        last = links[-1][1]
        cols = [g["cols"][j] for _, j in links] + g["cols"][last + 1:]
        rows = [g["rows"][i] for i, _ in links] + ["-"] * (len(g["cols"]) - last - 1)
        assert cols == g["alignment_cols"] and rows == g["alignment_rows"]
    if "marked_matches" in g:
        assert set(map(tuple, g["marked_matches"])) <= set(links)
        H, _, _ = oracle.nw(s, g["gap"])
        assert H[-1, -1] == g["nw_score"] < score


@pytest.mark.parametrize("seed", range(6))
def test_unconstrained_brute_force(seed):
    """The DP's optimum and path against every row-by-row choice (brute force)."""
    from oracle import unconstrained
    rng = np.random.default_rng(600 + seed)
    N, M = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    s = rng.random((N, M))
    p = float(rng.choice([0.05, 0.2, 0.4, 0.8]))
    scores = [_score_choice(s, p, ch) for ch in brute.unconstrained_choices(N, M)]
    best = max(scores)
    score, links = unconstrained.align(s, p)
    assert score == pytest.approx(best, abs=1e-12)
    choice = [None] * N
    for i, j in links:
        choice[i] = j
    assert _score_choice(s, p, choice) == pytest.approx(best, abs=1e-12)
    assert unconstrained.path_score(s, p, choice) == pytest.approx(best, abs=1e-12)


def test_unconstrained_without_the_move_back_is_nw():
    """Forbidding the move back leaves exactly Needleman-Wunsch: same optimum
    as the oracle's NW fill, and never better than the unconstrained one."""
    from oracle import unconstrained
    rng = np.random.default_rng(610)
    for _ in range(20):
        N, M = int(rng.integers(1, 9)), int(rng.integers(1, 9))
        s = rng.random((N, M))
        p = float(rng.choice([0.05, 0.3, 0.7]))
        H, _, diag = oracle.nw(s, p)
        score_nw, links = unconstrained.align(s, p, back=False)
        assert score_nw == pytest.approx(H[-1, -1], abs=1e-12)
        assert all(j2 > j1 for (_, j1), (_, j2) in zip(links, links[1:]))
        assert unconstrained.align(s, p)[0] >= score_nw - 1e-12


def test_unconstrained_single_column_closed_form():
    """M = 1: every row takes the column (matching again is a move back at
    cost p, never worse than leaving the row unmatched), so the optimum is
    s_0 + sum_{i>0} (s_i - p)."""
    from oracle import unconstrained
    rng = np.random.default_rng(611)
    s = rng.random((7, 1))
    p = 0.3
    score, links = unconstrained.align(s, p)
    assert score == pytest.approx(s[0, 0] + sum(s[i, 0] - p for i in range(1, 7)), abs=1e-12)
    assert links == [(i, 0) for i in range(7)]
