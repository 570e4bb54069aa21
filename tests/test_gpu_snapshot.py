"""The K-snapshot form on the GPU against the oracle's K-snapshot form.

In each block of K consecutive minibatches every minibatch steps from the
model as it stood when the block began and the changes are added in
minibatch order.  Bars as for Algorithm 1's order: parameters after a few
blocks within 1e-5 of the parameter scale, per-epoch train/test RMSE and MAE
within 1e-3 absolute; the combination order is fixed, so runs repeat bit for
bit.
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def synth():
    from paper_2012_03550_gb300 import synth as s
    return s


def _ctx(B, t, ranks, R, c, v, A0, B0, **opts):
    g = B.Tucker(t.shape, ranks, c, v, r_core=R, **opts)
    g.set_params(A0, B0, epoch=0)
    return g


def _params_case(B, synth, t, ranks, R, M, K, nb, lr, lam=(1e-3, 1e-3), init="normal", **opts):
    c, v = t.split("train")
    A0, B0 = synth.init_params(t.shape, ranks, R, mode=init, seed=1, mean_value=float(np.mean(v)))
    ref = O.Model(t.shape, ranks, R, A0, B0)
    ref.epoch_snapshot(c, v, M, 2, 0, K, lr[0], lr[1], lam[0], lam[1], 0, 0, nb)
    with _ctx(B, t, ranks, R, c, v, A0, B0, snapshot=K, **opts) as g:
        g.batches(lr[0], lr[1], lam[0], lam[1], M, 0, nb)
        Ag, Bg, core, _ = g.get_params()
    for n in range(len(ranks)):
        assert float(np.abs(Ag[n] - ref.A[n]).max()) <= 1e-5 * float(np.abs(ref.A[n]).max()), n
        assert float(np.abs(Bg[n] - ref.B[n]).max()) <= 1e-5 * float(np.abs(ref.B[n]).max()), n
    np.testing.assert_allclose(core, ref.build_core(), rtol=1e-4, atol=1e-5 * np.abs(ref.G).max())
    return Ag, Bg


@pytest.mark.parametrize("K", [4, 8])
def test_snapshot_params_rating_bench_minibatch(B, synth, K):
    # M = 4096 on the rating tensor's distributions: K groups of 152 / K CTAs
    # (K = 8: 216 samples per CTA), hot rows touched by every minibatch of a
    # block; the last block ragged
    w = synth.config2(scale=0.004)
    _params_case(B, synth, w.tensor, w.ranks, w.r_core, 4096, K, 2 * K + 3, (0.05, 0.05), init="rating")


def test_snapshot_params_config1_odd_k_and_short_last_block(B, synth):
    w = synth.config1()
    nb = (w.tensor.train.shape[0] + 255) // 256           # 176 minibatches: 58 blocks of 3 and one of 2
    _params_case(B, synth, w.tensor, w.ranks, 5, 256, 3, nb, (0.3, 0.2), (0.01, 0.02))


def test_snapshot_params_4order_and_kruskal_contraction(B, synth):
    w = synth.config3(scale=0.004)
    _params_case(B, synth, w.tensor, w.ranks, 5, 8192, 2, 6, (0.5, 0.5))
    t = synth.make_tensor((30, 20, 10, 8, 6), 2000, [("uniform",)] * 5, (2, 3, 2, 2, 3), 0.1, 0.0, seed=17)
    _params_case(B, synth, t, (2, 3, 2, 2, 3), 3, 64, 5, 31, (0.3, 0.2), contraction=1)


def test_snapshot_epoch_rmse_parity_fp32_and_bf16(B, synth):
    w = synth.config2(scale=0.004)
    t = w.tensor
    c, v = t.split("train")
    tc, tv = t.split("test")
    A0, B0 = synth.init_params(t.shape, w.ranks, w.r_core, mode="rating", seed=1, mean_value=float(np.mean(v)))
    ref = O.Model(t.shape, w.ranks, w.r_core, A0, B0)
    K, M, lr, lam = 4, 4096, 0.05, 1e-3
    worst = {0: 0.0, 1: 0.0}
    gs = {p: _ctx(B, t, w.ranks, w.r_core, c, v, A0, B0, snapshot=K, precision=p) for p in (0, 1)}
    try:
        for ep in range(4):
            ref.epoch_snapshot(c, v, M, 2, ep, K, lr, lr, lam, lam)
            for g in gs.values():
                g.epoch(lr, lr, lam, lam, M)
            for cc, vv in ((c, v), (tc, tv)):
                r_o, m_o = ref.rmse_mae(cc, vv)
                for p, g in gs.items():
                    r_g, m_g = g.rmse(cc, vv)
                    worst[p] = max(worst[p], abs(r_g - r_o), abs(m_g - m_o))
    finally:
        for g in gs.values():
            g.close()
    assert worst[0] <= 1e-3, worst
    assert worst[1] <= 1e-3, worst


def test_snapshot_runs_repeat_bit_for_bit(B, synth):
    w = synth.config2(scale=0.004)
    t = w.tensor
    c, v = t.split("train")
    A0, B0 = synth.init_params(t.shape, w.ranks, w.r_core, mode="rating", seed=1, mean_value=float(np.mean(v)))
    outs = []
    for _ in range(2):
        with _ctx(B, t, w.ranks, w.r_core, c, v, A0, B0, snapshot=4) as g:
            g.epoch(0.05, 0.05, 1e-3, 1e-3, 4096)
            outs.append(g.get_params())
    for x, y in zip(outs[0][0] + outs[0][1], outs[1][0] + outs[1][1]):
        assert np.array_equal(x, y)


def test_snapshot_rejects_what_it_cannot_run(B, synth):
    w = synth.config1()
    c, v = w.tensor.split("train")
    # K groups of ceil(M / 256) CTAs must fit on the GPU
    with B.Tucker(w.tensor.shape, w.ranks, c, v, r_core=5, snapshot=64) as g:
        with pytest.raises(B.StdError) as ei:
            g.epoch(0.1, 0.1, 1e-3, 1e-3, 4096)
        assert ei.value.code == B.STD_EUNSUPPORTED
    # batched launches run Algorithm 1's order only
    with B.Tucker(w.tensor.shape, w.ranks, c, v, r_core=5, snapshot=2) as g:
        with pytest.raises(B.StdError) as ei:
            B.std_batch_create([g.ctx], 0)
        assert ei.value.code == B.STD_EINVAL
