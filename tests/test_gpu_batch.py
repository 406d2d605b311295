"""Batched solves (swnmg_batch_*): every problem of a batch must end exactly
as its own single solve -- the same Newton and Step 1 sweep counts, the same
residual history and the same final state bit for bit -- whatever the batch's
mix of sizes and level counts, the CUDA-graph switch and the autotuner's
choices, and when other problems of the batch stop early or fail."""
import numpy as np
import pytest
import torch

from paper_1608_06721_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swnmg():
    from paper_1608_06721_gb300 import swnmg as S
    S.lib()
    return S


def _mixed_batch(precision):
    """Channels of several sizes, aspect ratios and level counts (the
    coarsest of each problem 8 x 8 or 8 x 4), W-cycles and exact coarsest
    solves as in the benchmark workloads."""
    specs = [(64, 64, 3, 11), (128, 32, 3, 12), (32, 32, 2, 13), (96, 64, 3, 14), (64, 128, 4, 15),
             (128, 128, 4, 16)]
    out = []
    for nx, ny, nl, seed in specs:
        p = W.channel_2d(seed=seed, nx=nx, ny=ny, n_levels=nl, precision=precision, redraw=False)
        out.append(p.with_params(gamma=2, eps_p=2.0, coarse_sweeps=0))
    return out


def _single(swnmg, p):
    S = swnmg.Solver(p)
    U = torch.as_tensor(np.ascontiguousarray(p.U0), dtype=torch.float64, device="cuda").contiguous()
    info = S.solve(U)
    return U.cpu().numpy(), info


def _same(info_b, info_s, Ub, Us):
    for k in ("status", "n_newton", "n_vcycles", "blusgs_sweeps", "init_res", "final_res", "res_hist"):
        assert info_b[k] == info_s[k], (k, info_b[k], info_s[k])
    assert np.array_equal(Ub, Us)


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_MIXED], ids=["fp64", "mixed"])
def test_batch_equals_single_solves(swnmg, precision):
    probs = _mixed_batch(precision)
    ref = [_single(swnmg, p) for p in probs]
    bt = swnmg.BatchSolver(probs)
    Us = bt.states()
    infos = bt.solve(Us)
    for p in range(len(probs)):
        _same(infos[p], ref[p][1], Us[p].cpu().numpy(), ref[p][0])
        assert infos[p]["status"] == 0


def test_batch_graph_and_tuning_do_not_change_results(swnmg):
    probs = _mixed_batch(W.PREC_MIXED)
    bt = swnmg.BatchSolver(probs)
    U0 = bt.states()
    base = [u.clone() for u in U0]
    info0 = bt.solve(base)
    chunks, blocks = bt.tune(bt.states())
    assert all(c in (4, 8, 16) for c in chunks) and min(blocks) > 0
    bt.set_graph(True)
    for ch, nb in ((chunks, 0), ([4] * 13, 38), ([8] * 13, max(blocks))):
        bt.set_tuning(ch, nb)
        Us = bt.states()
        infos = bt.solve(Us)
        for p in range(len(probs)):
            _same(infos[p], info0[p], Us[p].cpu().numpy(), base[p].cpu().numpy())
    # a second solve replays the captured graph
    Us = bt.states()
    infos = bt.solve(Us)
    for p in range(len(probs)):
        _same(infos[p], info0[p], Us[p].cpu().numpy(), base[p].cpu().numpy())


def test_failed_problem_does_not_disturb_the_others(swnmg):
    probs = _mixed_batch(W.PREC_FP64)[:4]
    ref = [_single(swnmg, p) for p in probs]
    bt = swnmg.BatchSolver(probs)
    Us = bt.states()
    Us[1][0, 5] = float("nan")
    infos = bt.solve(Us)
    assert infos[1]["status"] == swnmg.ERR_NONFINITE
    for p in (0, 2, 3):
        _same(infos[p], ref[p][1], Us[p].cpu().numpy(), ref[p][0])
    bad = bt.states()
    bad[1][0, 5] = float("nan")
    with pytest.raises(swnmg.SwnmgError) as e:
        bt.solve(bad, check=True)
    assert e.value.status == swnmg.ERR_NONFINITE


def test_batch_rejects_bad_input(swnmg):
    with pytest.raises(swnmg.SwnmgError) as e:
        swnmg.BatchSolver([W.subcritical_bump_1d(n=200)])
    assert e.value.status == swnmg.ERR_ARG
    p = W.channel_2d(nx=64, ny=64, n_levels=1, redraw=False).with_params(coarse_sweeps=0)
    with pytest.raises(swnmg.SwnmgError) as e:   # 32 x 32 coarsest: no guarded inverse, no sweeps
        swnmg.BatchSolver([p])
    assert e.value.status == swnmg.ERR_ARG
    bt = swnmg.BatchSolver(_mixed_batch(W.PREC_MIXED)[:2])
    with pytest.raises(swnmg.SwnmgError):
        bt.set_tuning([3] * 13)
    with pytest.raises(swnmg.SwnmgError):
        bt.set_tuning(None, 1 << 20)


def test_batch_with_coarse_sweeps(swnmg):
    """coarse_sweeps > 0: every problem's coarsest level is smoothed instead."""
    probs = [p.with_params(coarse_sweeps=4) for p in _mixed_batch(W.PREC_FP64)[:3]]
    ref = [_single(swnmg, p) for p in probs]
    bt = swnmg.BatchSolver(probs)
    Us = bt.states()
    infos = bt.solve(Us)
    for p in range(len(probs)):
        _same(infos[p], ref[p][1], Us[p].cpu().numpy(), ref[p][0])


def test_batched_channel_workload_subset(swnmg):
    """Problems of the batched workload recipe (the 128 x 128 and 256 x 256
    ones among its first 16) against their single solves."""
    probs = [p for p in W.batch_channels(count=16) if p.nx <= 256][:6]
    assert len(probs) >= 3
    ref = [_single(swnmg, p) for p in probs]
    bt = swnmg.BatchSolver(probs)
    bt.tune(bt.states())
    bt.set_graph(True)
    Us = bt.states()
    infos = bt.solve(Us)
    for p in range(len(probs)):
        _same(infos[p], ref[p][1], Us[p].cpu().numpy(), ref[p][0])


def test_batch_eps_p_rule_per_problem(swnmg):
    """eps_p < 0 (the paper's rule) gives every problem of a batch its own
    Step 1 thresholds from its own initial residual: each problem still ends
    exactly as its single solve."""
    probs = [p.with_params(eps_p=-0.01) for p in _mixed_batch(W.PREC_MIXED)]
    ref = [_single(swnmg, p) for p in probs]
    bt = swnmg.BatchSolver(probs)
    Us = bt.states()
    infos = bt.solve(Us)
    for p in range(len(probs)):
        _same(infos[p], ref[p][1], Us[p].cpu().numpy(), ref[p][0])
