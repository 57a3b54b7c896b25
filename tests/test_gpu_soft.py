"""GPU parity of the soft (differentiable) alignment against the FP64 oracle.

Tolerances (FP32 kernels vs FP64 oracle):
  soft value V(N,M)     |dV| <= 1e-4 * max(1, |V|)
  expected alignment E  |dE| <= 2e-4 (gamma 1, 0.1), 2e-3 (gamma 0.01)
  loss                  relative 1e-4
  gradients             relative 1e-3 of the largest component (FP32 GPU vs
                        FP64 oracle); the oracle's own gradient is pinned to
                        central differences in tests/test_oracle.py
"""
import numpy as np
import pytest

import oracle
from paper_1512_01641_gb300 import synth

pytestmark = pytest.mark.gpu

THETA = np.array([4.0, 4.0, -2.0, 1.0, -3.0, 0.3, 0.5])
TAU = 0.05


def _batch(seed, n_pairs, n, v=400):
    return synth.make_batch(seed, n_pairs, v_src=v, v_tgt=v, planted_frac=1.0, src_sizes=np.full(n_pairs, n))


def _gpu_soft(batch, gamma, theta=THETA, want=True):
    import torch
    from paper_1512_01641_gb300 import miner
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    counts = plan.count()
    gold = torch.from_numpy(miner.gold_cells(batch, plan)).cuda()
    al = miner.SoftAligner(plan, counts, gold, gamma, TAU)
    params = miner.params_from_theta(theta)
    loss, value, exp = al.forward(params, want_value=want, want_expected=want)
    grad = al.backward(params)
    plan.check()
    torch.cuda.synchronize()
    return {"plan": plan, "loss": float(loss[0]), "value": value.cpu().numpy() if want else None,
            "E": exp.cpu().numpy() if want else None, "grad": grad.cpu().numpy().astype(np.float64),
            "aligner": al, "counts": counts}


def _oracle_pairs(batch, theta=THETA):
    r = oracle.mine(batch, theta[:4], theta[4], theta[5], theta[6], want_counts=True, want_sim=True)
    pairs = []
    for k in range(batch.n_pairs):
        c = r["counts"][k]
        ls = [len(x) for x in batch.src.doc(k)]
        lt = [len(x) for x in batch.tgt.doc(k)]
        gold = np.zeros(c.shape[:2])
        for i, j in batch.gold[k]:
            gold[i, j] = 1
        pairs.append((c[..., 0], c[..., 1], ls, lt, gold))
    return r, pairs


@pytest.mark.parametrize("gamma", [1.0, 0.1, 0.01])
def test_soft_value_and_expected_alignment(gamma):
    batch = _batch(301, 6, 45)
    g = _gpu_soft(batch, gamma)
    r, _ = _oracle_pairs(batch)
    off = g["plan"].cell_offsets
    etol = 2e-3 if gamma < 0.05 else 2e-4
    for k in range(batch.n_pairs):
        V, E, dp = oracle.soft_nw(r["sim"][k], THETA[5], gamma)
        assert abs(g["value"][k] - V[-1, -1]) <= 1e-4 * max(1.0, abs(V[-1, -1])), (k, g["value"][k], V[-1, -1])
        Eg = g["E"][off[k]:off[k + 1]].reshape(E.shape)
        assert np.abs(Eg - E).max() <= etol, (k, np.abs(Eg - E).max())


@pytest.mark.parametrize("gamma", [1.0, 0.1, 0.01])
def test_soft_loss_and_gradient_vs_oracle(gamma):
    pytest.importorskip("torch")
    from oracle import softgrad
    batch = _batch(302, 4, 10)
    g = _gpu_soft(batch, gamma)
    _, pairs = _oracle_pairs(batch)
    L, grad = softgrad.loss_and_grad(pairs, THETA, gamma, TAU)
    assert g["loss"] == pytest.approx(L, rel=1e-4)
    scale = np.abs(grad).max()
    assert np.abs(g["grad"] - grad).max() <= 1e-3 * scale, (g["grad"], grad)


def test_soft_gradient_vs_central_differences_16_pairs_8x8():
    """GPU backward against FP64 central differences (h = 1e-6) of the oracle
    loss, 16 pairs of 8 x 8 sentences."""
    pytest.importorskip("torch")
    from oracle import softgrad
    batch = synth.make_batch(303, 16, v_src=300, v_tgt=300, planted_frac=1.0, src_sizes=np.full(16, 8),
                             p_sdrop=0.0, p_ins=0.0)
    assert np.all(batch.tgt.doc_sizes() == 8)
    gamma = 0.1
    g = _gpu_soft(batch, gamma, want=False)
    _, pairs = _oracle_pairs(batch)
    h = 1e-6
    fd = np.zeros(7)
    for k in range(7):
        tp, tm = THETA.copy(), THETA.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (softgrad.loss_value(pairs, tp, gamma, TAU) - softgrad.loss_value(pairs, tm, gamma, TAU)) / (2 * h)
    assert np.abs(g["grad"] - fd).max() <= 1e-3 * np.abs(fd).max(), (g["grad"], fd)


def test_autograd_function_matches_kernels():
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _batch(304, 5, 30)
    g = _gpu_soft(batch, 0.1, want=False)
    theta = torch.tensor(THETA, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = miner.soft_nw_loss(theta, g["aligner"])
    loss.backward()
    assert float(loss) == pytest.approx(g["loss"], rel=1e-6)
    assert np.allclose(theta.grad.cpu().numpy(), g["grad"], rtol=1e-6, atol=0)


def test_soft_tends_to_hard_alignment():
    """At small gamma the expected alignment concentrates on the hard path."""
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _batch(305, 4, 40)
    g = _gpu_soft(batch, 0.002)
    plan = g["plan"]
    out = plan.align(miner.params_from_theta(THETA[:6].tolist() + [-1.0]), g["counts"])
    links = miner.links_per_pair(out, batch.n_pairs)
    off = plan.cell_offsets
    M = batch.tgt.doc_sizes()
    on_path = []
    for k in range(batch.n_pairs):
        E = g["E"][off[k]:off[k + 1]].reshape(-1, M[k])
        on_path += [E[i, j] for i, j, _ in links[k]]
        # E is a distribution over paths: every diagonal count is at most 1
        assert E.min() >= -1e-6 and E.sum(axis=0).max() <= 1 + 1e-4 and E.sum(axis=1).max() <= 1 + 1e-4
    assert np.mean(np.array(on_path) > 0.9) >= 0.95


@pytest.mark.parametrize("gamma", [1.0, 0.1])
def test_soft_hessian_vector_product_per_cell(gamma):
    """H u per cell (the derivative of E along u = dL/dE) against the oracle's
    FP64 double-backward.  At gamma 0.1 these clean 8 x 8 pairs are saturated
    (|H u| ~ 1e-5 |u|): the error bound is relative to |H u| itself, which only
    holds because the tangent differences are formed without cancellation."""
    pytest.importorskip("torch")
    from oracle import softgrad
    from paper_1512_01641_gb300 import miner
    batch = synth.make_batch(306, 3, v_src=300, v_tgt=300, planted_frac=1.0, src_sizes=np.full(3, 8),
                             p_sdrop=0.0, p_ins=0.0)
    g = _gpu_soft(batch, gamma, want=False)
    _, hu = g["aligner"].backward(miner.params_from_theta(THETA), want_hvp=True)
    hu = hu.cpu().numpy()
    _, pairs = _oracle_pairs(batch)
    off = g["plan"].cell_offsets
    n_cells = g["plan"].n_cells
    for k, pr in enumerate(pairs):
        E, u, h = softgrad.hvp_cells(*pr, THETA, gamma, TAU, n_cells)
        got = hu[off[k]:off[k + 1]].reshape(h.shape)
        err = np.abs(got - h).max()
        print(f"pair {k}: max|u| {np.abs(u).max():.3e} max|Hu| {np.abs(h).max():.3e} err {err:.3e} "
              f"sum Hu gpu {got.sum():.6e} oracle {h.sum():.6e}")
        assert err <= 1e-4 * np.abs(h).max()
        assert abs(got.sum() - h.sum()) <= 1e-4 * np.abs(h).sum()


def test_minibatch_selection_equals_plan_of_the_subset():
    """A selected subset of pairs gives the loss and gradient of a plan built
    from just those pairs (the mean runs over the selected cells)."""
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _batch(307, 12, 20)
    pick = np.array([3, 7, 0, 10, 5])
    full = _gpu_soft(batch, 0.1, want=False)
    al = full["aligner"]
    al.select(pick)
    params = miner.params_from_theta(THETA)
    loss, _, _ = al.forward(params)
    grad = al.backward(params).cpu().numpy()
    sub = _gpu_soft(batch.subset(np.sort(pick)), 0.1, want=False)
    assert float(loss[0]) == pytest.approx(sub["loss"], rel=1e-5)
    assert np.allclose(grad, sub["grad"], rtol=1e-4, atol=1e-7 * np.abs(sub["grad"]).max())
    al.select(None)
    loss_all, _, _ = al.forward(params)
    assert float(loss_all[0]) == pytest.approx(full["loss"], rel=1e-6)


def _soft_all(plan, counts, gold, gamma, split):
    from paper_1512_01641_gb300 import miner
    plan.set_option("soft_split", split)
    al = miner.SoftAligner(plan, counts, gold, gamma, TAU)
    params = miner.params_from_theta(THETA)
    loss, value, exp = al.forward(params, want_value=True, want_expected=True)
    grad, hvp = al.backward(params, want_hvp=True)
    plan.check()
    return [x.cpu().numpy().copy() for x in (loss, value, exp, grad, hvp)]


def test_split_sweeps_are_bit_identical_to_one_warp_per_pair():
    """Splitting a pair's strips over warps (a wavefront with progress
    counters) runs the same arithmetic in the same order: loss, V, E, the
    gradient and H u are bit-identical in all four modes, on pairs of 1 to
    9 strips with ragged last strips and ragged column blocks."""
    import torch
    from paper_1512_01641_gb300 import miner
    sizes = np.array([5, 33, 70, 150, 260, 64, 31, 97])
    batch = synth.make_batch(308, len(sizes), v_src=500, v_tgt=500, planted_frac=1.0, src_sizes=sizes)
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    counts = plan.count()
    gold = torch.from_numpy(miner.gold_cells(batch, plan)).cuda()
    ref = _soft_all(plan, counts, gold, 0.1, 0)
    for split in (1, 2, 3):
        got = _soft_all(plan, counts, gold, 0.1, split)
        for name, a, b in zip(("loss", "value", "E", "grad", "hvp"), ref, got):
            assert np.array_equal(a, b), (split, name, np.abs(a - b).max())
    assert plan.get_option("soft_split") == 3
    # mode 1 with other split thresholds (quarters of the mean chain per warp)
    for q4 in (1, 64):
        plan.set_option("soft_split_q4", q4)
        for split in (1, 3):
            got = _soft_all(plan, counts, gold, 0.1, split)
            for name, a, b in zip(("loss", "value", "E", "grad", "hvp"), ref, got):
                assert np.array_equal(a, b), (q4, split, name, np.abs(a - b).max())
    assert plan.get_option("soft_split_q4") == 64
    # the other work-list orders (value sweeps and adjoints per pair; adjoints before whole pairs)
    plan.set_option("soft_split_q4", 4)
    for order in (0, 2):
        plan.set_option("soft_order", order)
        for split in (1, 2):
            got = _soft_all(plan, counts, gold, 0.1, split)
            for name, a, b in zip(("loss", "value", "E", "grad", "hvp"), ref, got):
                assert np.array_equal(a, b), (order, split, name, np.abs(a - b).max())


def test_split_sweep_multi_strip_pair_vs_oracle():
    """A 9-strip pair swept as a wavefront over nine warps (split mode 2):
    V and E against the FP64 oracle."""
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _batch(309, 2, 270, v=600)
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    counts = plan.count()
    gold = torch.from_numpy(miner.gold_cells(batch, plan)).cuda()
    _, value, E, _, _ = _soft_all(plan, counts, gold, 0.1, 2)
    r, _ = _oracle_pairs(batch)
    off = plan.cell_offsets
    for k in range(batch.n_pairs):
        Vo, Eo, _ = oracle.soft_nw(r["sim"][k], THETA[5], 0.1)
        assert abs(value[k] - Vo[-1, -1]) <= 1e-4 * max(1.0, abs(Vo[-1, -1]))
        assert np.abs(E[off[k]:off[k + 1]].reshape(Eo.shape) - Eo).max() <= 2e-4


@pytest.mark.slow
@pytest.mark.parametrize("gamma", [1.0, 0.1, 0.01])
def test_soft_full_size_4096_pairs_sampled(gamma):
    """The soft configuration at full size (4,096 planted pairs of ~100 x 100
    sentences, the long ones split over warps): soft V(N,M) and the expected
    alignment E of 24 sampled pairs against the FP64 oracle."""
    import torch
    from paper_1512_01641_gb300 import miner
    batch = synth.soft_batch()
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    counts = plan.count()
    gold = torch.from_numpy(miner.gold_cells(batch, plan)).cuda()
    al = miner.SoftAligner(plan, counts, gold, gamma, TAU)
    params = miner.params_from_theta(THETA)
    _, value, exp = al.forward(params, want_value=True, want_expected=True)
    plan.check()
    sizes = batch.src.doc_sizes() * batch.tgt.doc_sizes()
    rng = np.random.default_rng(9)
    pick = np.unique(np.concatenate([np.argsort(sizes)[-4:], rng.choice(batch.n_pairs, 20, replace=False)]))
    sub = batch.subset(pick)
    r = oracle.mine(sub, THETA[:4], THETA[4], THETA[5], THETA[6], want_sim=True)
    off = plan.cell_offsets
    etol = 2e-3 if gamma < 0.05 else 2e-4
    for x, k in enumerate(pick):
        V, E, _ = oracle.soft_nw(r["sim"][x], THETA[5], gamma)
        v = float(value[k])
        assert abs(v - V[-1, -1]) <= 1e-4 * max(1.0, abs(V[-1, -1])), (k, v, V[-1, -1])
        Eg = exp[off[k]:off[k + 1]].cpu().numpy().reshape(E.shape)
        assert np.abs(Eg - E).max() <= etol, (k, np.abs(Eg - E).max())
    plan.close()


@pytest.mark.parametrize("gamma", [1.0, 0.1])
def test_multi_strip_backward_vs_oracle(gamma):
    """The strip-recompute backward on pairs of two to four 32-row strips
    (ragged last strips and ragged column blocks): the 7 gradients and H u of
    every cell against the FP64 oracle's double backward, with the strips on
    one warp (split mode 0) and every strip on its own warp (split mode 2)."""
    pytest.importorskip("torch")
    import torch
    from oracle import softgrad
    from paper_1512_01641_gb300 import miner
    ns, ms = [40, 70, 97], [45, 33, 64]
    batch = synth.make_batch(310, 3, v_src=500, v_tgt=500, planted_frac=0.0, src_sizes=ns, tgt_sizes=ms)
    # planted-like gold on the diagonal band, so the loss has both kinds of cells
    batch.gold = [np.array([(i, int(i * m / n)) for i in range(n)], np.int32) for n, m in zip(ns, ms)]
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    counts = plan.count()
    gold = torch.from_numpy(miner.gold_cells(batch, plan)).cuda()
    _, pairs = _oracle_pairs(batch)
    L, grad = softgrad.loss_and_grad(pairs, THETA, gamma, TAU)
    n_cells = plan.n_cells
    hu_o = [softgrad.hvp_cells(*pr, THETA, gamma, TAU, n_cells)[2] for pr in pairs]
    off = plan.cell_offsets
    for split in (0, 2):
        loss, _, _, g, hu = _soft_all(plan, counts, gold, gamma, split)
        assert float(loss[0]) == pytest.approx(L, rel=1e-4), split
        g = g.astype(np.float64)
        assert np.abs(g - grad).max() <= 1e-3 * np.abs(grad).max(), (split, g, grad)
        for k, h in enumerate(hu_o):
            got = hu[off[k]:off[k + 1]].reshape(h.shape)
            assert np.abs(got - h).max() <= 1e-4 * np.abs(h).max(), (split, k, np.abs(got - h).max())
    plan.close()


def test_soft_split_wait_reports_timeout_and_recovers():
    """A strip's forward progress counter that nothing publishes (fault
    injection) in a pair split over warps: the strips that wait on it give up
    after a short bounded poll, mine_plan_check reports MINE_ETIMEOUT, the
    context stays usable, and the next normal call is correct."""
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _batch(311, 1, 100, v=500)
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    counts = plan.count()
    gold = torch.from_numpy(miner.gold_cells(batch, plan)).cuda()
    ref = _soft_all(plan, counts, gold, 0.1, 2)
    plan.set_option("wait_limit", 2000)
    plan.set_option("fault_skip_soft", 0)
    al = miner.SoftAligner(plan, counts, gold, 0.1, TAU)
    al.forward(miner.params_from_theta(THETA))
    with pytest.raises(miner.MinerError) as e:
        plan.check()
    assert e.value.code == miner.MINE_ETIMEOUT
    plan.set_option("fault_skip_soft", -1)
    plan.set_option("wait_limit", 1 << 24)
    got = _soft_all(plan, counts, gold, 0.1, 2)
    for name, a, b in zip(("loss", "value", "E", "grad", "hvp"), ref, got):
        assert np.array_equal(a, b), name
    assert plan.get_option("fault_skip_soft") == -1
    plan.close()
