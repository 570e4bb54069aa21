"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: sampled indices, sort permutations and run boundaries bit-exact;
one minibatch's core and factor gradients within 1e-5 relative in FP32,
norm-wise over each mode's gradient (FP32 residuals x-hat - x lose relative
accuracy when x-hat is close to x, so single small rows are held to a mixed
relative/absolute bound instead); per-epoch train/test RMSE within 1e-3 absolute over
10 epochs.  Parameters after a step are compared with a tolerance derived from
FP32 rounding of the same arithmetic (1e-5 relative to the parameter scale).
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


@pytest.fixture(scope="module")
def cfg1(synth):
    return synth.config1()


def _gpu(B, shape, ranks, R, coords, vals, A0=None, B0=None, **opts):
    t = B.Tucker(shape, ranks, coords, vals, r_core=R, **opts)
    if A0 is not None:
        t.set_params(A0, B0, epoch=0)
    return t


def _rel(a, b):
    d = float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)))
    s = float(np.linalg.norm(np.asarray(b, np.float64)))
    return d / s if s > 0 else d


# ---------------------------------------------------------------------------
# Sampler + tiler: bit-exact
# ---------------------------------------------------------------------------

def _check_schedule(B, gpu, coords, M, batches, seed=2, epoch=0):
    n = coords.shape[0]
    sid, order, s0, s1 = gpu.schedule(M, batches[0], batches[1])
    t0 = batches[0] * M
    ref = O.perm_range(n, seed, epoch, t0, sid.shape[0])
    assert np.array_equal(sid.astype(np.int64), ref)
    for b in range(batches[0], batches[1]):
        lo, hi = b * M - t0, min((b + 1) * M, n) - t0
        ids = ref[lo:hi]
        for mode in range(coords.shape[1]):
            keys = coords[ids, mode]
            o_ref, seg = O.stable_order(keys)
            assert np.array_equal(order[mode, lo:hi], o_ref)
            st = np.repeat(seg[:-1], np.diff(seg))
            en = np.repeat(seg[1:] - 1, np.diff(seg))
            assert np.array_equal(s0[mode, lo:hi], st)
            assert np.array_equal(s1[mode, lo:hi], en)


def test_schedule_bitexact_uniform(B, cfg1):
    c, v = cfg1.tensor.split("train")
    with B.Tucker(cfg1.tensor.shape, cfg1.ranks, c, v, r_core=5) as g:
        nb = (c.shape[0] + 255) // 256
        _check_schedule(B, g, c, 256, (0, nb))


@pytest.mark.parametrize("M", [1, 7, 4096, 8192])
def test_schedule_bitexact_zipf_ragged(B, synth, M):
    # rating-like, Zipf-hot rows (long runs), ragged last minibatch
    t = synth.make_tensor((5000, 800, 60), 50_001, [("zipf", 1.1), ("zipf", 1.3), ("uniform",)],
                          (4, 4, 4), 0.1, 0.0, seed=9)
    c, v = t.split("train")
    with B.Tucker(t.shape, (4, 4, 4), c, v, r_core=2) as g:
        nb = (c.shape[0] + M - 1) // M
        rng = (0, nb) if M >= 4096 else (nb - 3, nb)
        _check_schedule(B, g, c, M, rng)


# ---------------------------------------------------------------------------
# Prediction and RMSE/MAE
# ---------------------------------------------------------------------------

def test_predict_and_rmse_parity(B, synth, cfg1):
    c, v = cfg1.tensor.split("train")
    tc, tv = cfg1.tensor.split("test")
    A0, B0 = synth.init_params(cfg1.tensor.shape, cfg1.ranks, 5, mode="normal", seed=1)
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0) as g:
        ref = O.Model(cfg1.tensor.shape, cfg1.ranks, 5, A0, B0)
        got = g.predict(tc)
        want = ref.predict(tc)
        np.testing.assert_allclose(got, want, rtol=2e-5, atol=2e-6 * np.abs(want).max())
        r, a = g.rmse(tc, tv)
        rr, ra = ref.rmse_mae(tc, tv)
        assert abs(r - rr) <= 1e-5 * rr and abs(a - ra) <= 1e-5 * ra
        # k = 0 and the fixed reduction order are deterministic
        assert g.rmse(tc[:0], tv[:0]) == (0.0, 0.0)
        assert g.rmse(tc, tv) == (r, a)


def test_predict_rejects_out_of_range(B, cfg1):
    c, v = cfg1.tensor.split("train")
    with B.Tucker(cfg1.tensor.shape, cfg1.ranks, c, v, r_core=5) as g:
        bad = np.array([[0, 0, 0], [500, 0, 0]], np.int32)
        with pytest.raises(B.StdError) as ei:
            g.predict(bad)
        assert ei.value.code == B.STD_EINVAL
        # the context stays usable
        assert np.isfinite(g.predict(bad[:1])).all()


def test_create_rejects_out_of_range_index(B):
    coords = np.array([[0, 0, 0], [1, 9, 0]], np.int32)
    vals = np.ones(2, np.float32)
    with pytest.raises(B.StdError) as ei:
        B.Tucker((4, 4, 4), (2, 2, 2), coords, vals, r_core=2)
    assert ei.value.code == B.STD_EINVAL


# ---------------------------------------------------------------------------
# One minibatch: gradients and parameters
# ---------------------------------------------------------------------------

def _step_case(B, synth, tensor, ranks, R, M, batch, lr=(0.3, 0.2), lam=(0.01, 0.02), norm_mode=0, init="normal",
               **opts):
    """Probe minibatch `batch` of epoch 0 from one state on both sides.  For
    batch > 0 the state is the oracle's FP64 state after batches [0, batch),
    rounded to FP32 and given to both sides (a one-step comparison)."""
    c, v = tensor.split("train")
    A0, B0 = synth.init_params(tensor.shape, ranks, R, mode=init, seed=1,
                               mean_value=float(np.mean(v)))
    if batch > 0:
        adv = O.Model(tensor.shape, ranks, R, A0, B0)
        adv.epoch(c, v, M, 2, 0, lr[0], lr[1], lam[0], lam[1], norm_mode, 0, batch)
        A0 = [a.astype(np.float32) for a in adv.A]
        B0 = [b.astype(np.float32) for b in adv.B]
    ref = O.Model(tensor.shape, ranks, R, A0, B0)
    with _gpu(B, tensor.shape, ranks, R, c, v, A0, B0, norm_mode=norm_mode, **opts) as g:
        sched = O.perm_range(c.shape[0], 2, 0, batch * M, min(M, c.shape[0] - batch * M))
        pr = g.batches(lr[0], lr[1], lam[0], lam[1], M, batch, batch + 1, probe=True)
        V, F, nseg = ref.step(c[sched], v[sched], lr[0], lr[1], lam[0], lam[1], norm_mode=norm_mode, probe=True)
        Ag, Bg, core, _ = g.get_params()
    # Norm-wise relative error of each mode's gradient (all R columns of B(n);
    # all touched rows of A(n)); each row also within a mixed bound so a
    # single wrong row cannot hide in the norm.
    N = len(ranks)
    worst_v = worst_f = 0.0
    for n in range(N):
        Jn = ranks[n]
        worst_v = max(worst_v, _rel(pr["core_V"][n, :R, :Jn], V[n, :R, :Jn]))
        assert pr["nseg"][n] == nseg[n]
        U = int(nseg[n])
        Fg, Fo = pr["factor_F"][n, :U, :Jn], F[n, :U, :Jn]
        worst_f = max(worst_f, _rel(Fg, Fo))
        row_err = np.linalg.norm(Fg - Fo, axis=1)
        row_tol = 1e-5 * np.linalg.norm(Fo, axis=1) + 1e-6 * np.linalg.norm(Fo, axis=1).max()
        assert np.all(row_err <= row_tol), float((row_err / row_tol).max())
    assert worst_v <= 1e-5, worst_v
    assert worst_f <= 1e-5, worst_f
    for n in range(N):
        sa = float(np.abs(ref.A[n]).max())
        sb = float(np.abs(ref.B[n]).max())
        assert float(np.abs(Ag[n] - ref.A[n]).max()) <= 1e-5 * sa
        assert float(np.abs(Bg[n] - ref.B[n]).max()) <= 1e-5 * sb
    np.testing.assert_allclose(core, ref.build_core(), rtol=1e-4, atol=1e-5 * np.abs(ref.G).max())
    return worst_v, worst_f


def test_step_gradients_config1(B, synth, cfg1):
    _step_case(B, synth, cfg1.tensor, cfg1.ranks, 5, 256, batch=0)


def test_step_gradients_config1_later_batch_and_last(B, synth, cfg1):
    _step_case(B, synth, cfg1.tensor, cfg1.ranks, 5, 256, batch=3)
    nb = (cfg1.tensor.train.shape[0] + 255) // 256
    _step_case(B, synth, cfg1.tensor, cfg1.ranks, 5, 256, batch=nb - 1)


def test_step_gradients_rating_zipf_4096(B, synth):
    # Netflix-like distributions scaled down: hot rows span many CTA chunks
    w = synth.config2(scale=0.004)
    _step_case(B, synth, w.tensor, w.ranks, 5, 4096, batch=1, init="rating", lr=(0.05, 0.05))


def test_step_gradients_4order_8192(B, synth):
    w = synth.config3(scale=0.004)
    _step_case(B, synth, w.tensor, w.ranks, 5, 8192, batch=0)


@pytest.mark.parametrize("norm_mode", [1])
def test_step_gradients_row_count_normaliser(B, synth, cfg1, norm_mode):
    _step_case(B, synth, cfg1.tensor, cfg1.ranks, 5, 256, batch=2, norm_mode=norm_mode)


@pytest.mark.parametrize("shape,ranks,R,M,nnz", [
    ((50, 40), (3, 5), 2, 17, 300),              # N = 2
    ((30, 20, 10, 8, 6), (2, 3, 2, 2, 3), 3, 64, 2000),   # N = 5, mixed ranks
    ((9, 8, 7), (1, 1, 1), 1, 1, 40),             # rank 1, M = 1
    ((12, 11, 10), (6, 5, 4), 7, 500, 333),       # one short minibatch (M > nnz)
])
def test_step_gradients_edge_shapes(B, synth, shape, ranks, R, M, nnz):
    t = synth.make_tensor(shape, nnz, [("uniform",)] * len(shape), ranks, 0.1, 0.0, seed=17)
    _step_case(B, synth, t, ranks, R, M, batch=0)


# The rank-sweep extremes of the paper's parameter study: a wide mode (J_1 =
# 25, the largest Kronecker rows and Gram blocks) and a wide core (R_core =
# 25, 300 Gram blocks and 25 cyclic steps per mode).
@pytest.mark.parametrize("ranks,R", [((25, 5, 5), 5), ((5, 5, 5), 25), ((15, 5, 5), 5)])
def test_step_gradients_rank_sweep_points(B, synth, ranks, R):
    t = synth.make_tensor((300, 200, 100), 6000, [("zipf", 1.1), ("zipf", 1.3), ("uniform",)], (5, 5, 5),
                          0.05, 0.0, seed=23)
    _step_case(B, synth, t, ranks, R, 2048, batch=1, lr=(0.05, 0.05))


def test_epoch_rmse_parity_rank_sweep_wide_core(B, synth):
    t = synth.make_tensor((300, 200, 100), 6000, [("zipf", 1.1), ("zipf", 1.3), ("uniform",)], (5, 5, 5),
                          0.05, 0.1, seed=29)
    ranks, R, M, lr, lam = (5, 5, 5), 25, 512, 0.01, 1e-3
    c, v = t.split("train")
    tc, tv = t.split("test")
    A0, B0 = synth.init_params(t.shape, ranks, R, mode="normal", seed=1)
    ref = O.Model(t.shape, ranks, R, A0, B0)
    worst = 0.0
    with _gpu(B, t.shape, ranks, R, c, v, A0, B0) as g:
        for ep in range(3):
            g.epoch(lr, lr, lam, lam, M)
            ref.epoch(c, v, M, 2, ep, lr, lr, lam, lam)
            for cc, vv in ((c, v), (tc, tv)):
                r_g, m_g = g.rmse(cc, vv)
                r_o, m_o = ref.rmse_mae(cc, vv)
                worst = max(worst, abs(r_g - r_o), abs(m_g - m_o))
    assert worst <= 1e-3, worst


# The Kruskal form of the factor-phase contraction (E_s = B(n) w_s) is the
# same product as the Kronecker rows against the unfolded core (Eq. 4 in
# Eq. 11), so it is held to the same bars against the same oracle.
def test_step_gradients_kruskal_contraction_config1(B, synth, cfg1):
    _step_case(B, synth, cfg1.tensor, cfg1.ranks, 5, 256, batch=0, contraction=1)


def test_step_gradients_kruskal_contraction_rating_zipf(B, synth):
    w = synth.config2(scale=0.004)
    _step_case(B, synth, w.tensor, w.ranks, 5, 4096, batch=1, init="rating", lr=(0.05, 0.05), contraction=1)


def test_step_gradients_kruskal_contraction_4order_and_edge(B, synth):
    w = synth.config3(scale=0.004)
    _step_case(B, synth, w.tensor, w.ranks, 5, 8192, batch=0, contraction=1)
    t = synth.make_tensor((30, 20, 10, 8, 6), 2000, [("uniform",)] * 5, (2, 3, 2, 2, 3), 0.1, 0.0, seed=17)
    _step_case(B, synth, t, (2, 3, 2, 2, 3), 3, 64, batch=0, contraction=1)


def test_epoch_rmse_parity_kruskal_contraction(B, synth, cfg1):
    c, v = cfg1.tensor.split("train")
    tc, tv = cfg1.tensor.split("test")
    A0, B0 = synth.init_params(cfg1.tensor.shape, cfg1.ranks, 5, mode="normal", seed=1)
    ref = O.Model(cfg1.tensor.shape, cfg1.ranks, 5, A0, B0)
    worst = 0.0
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0, contraction=1) as g:
        for ep in range(4):
            g.epoch(0.5, 0.5, cfg1.lam, cfg1.lam, cfg1.minibatch)
            ref.epoch(c, v, cfg1.minibatch, 2, ep, 0.5, 0.5, cfg1.lam, cfg1.lam)
            r_g, m_g = g.rmse(tc, tv)
            r_o, m_o = ref.rmse_mae(tc, tv)
            worst = max(worst, abs(r_g - r_o), abs(m_g - m_o))
    assert worst <= 1e-3, worst


# The paper's own setting (Sec. 5.1, 5.3): initialisation N(0.5, 0.1^2),
# gamma_A = 0.002, gamma_B = 0.001, lambda_A = lambda_B = 0.01, one sample per
# step (M = 1), the row's sample count as normaliser, and B updated only in
# the first and the last epoch (lr_b = 0 in between leaves B untouched).
def test_paper_setting_m1_core_schedule(B, synth):
    t = synth.make_tensor((60, 50, 40), 1500, [("uniform",)] * 3, (5, 5, 5), 0.05, 0.1, seed=31)
    ranks, R = (5, 5, 5), 5
    c, v = t.split("train")
    tc, tv = t.split("test")
    A0, B0 = synth.init_params(t.shape, ranks, R, mode="paper", seed=1)
    ref = O.Model(t.shape, ranks, R, A0, B0)
    epochs, ga, gb, lam = 4, 0.002, 0.001, 0.01
    worst = 0.0
    with _gpu(B, t.shape, ranks, R, c, v, A0, B0, norm_mode=1) as g:
        for ep in range(epochs):
            lr_b = gb if ep in (0, epochs - 1) else 0.0
            _, Bb, _, _ = g.get_params()
            g.epoch(ga, lr_b, lam, lam, 1)
            ref.epoch(c, v, 1, 2, ep, ga, lr_b, lam, lam, 1)
            Ag, Ba, _, _ = g.get_params()
            if lr_b == 0.0:
                for n in range(3):
                    assert np.array_equal(Ba[n], Bb[n])   # B untouched, bit for bit
            r_g, m_g = g.rmse(tc, tv)
            r_o, m_o = ref.rmse_mae(tc, tv)
            worst = max(worst, abs(r_g - r_o), abs(m_g - m_o))
            for n in range(3):
                assert float(np.abs(Ag[n] - ref.A[n]).max()) <= 1e-4 * float(np.abs(ref.A[n]).max())
    assert worst <= 1e-3, worst


# Heavy-ball momentum (the accelerated SGD the paper names as future work):
# several consecutive minibatches, so that the velocities carry over, against
# the oracle with the same momentum.
@pytest.mark.parametrize("mu,precision_args", [(0.9, {}), (0.5, {"contraction": 1})])
def test_momentum_consecutive_minibatches(B, synth, cfg1, mu, precision_args):
    c, v = cfg1.tensor.split("train")
    A0, B0 = synth.init_params(cfg1.tensor.shape, cfg1.ranks, 5, mode="normal", seed=1)
    ref = O.Model(cfg1.tensor.shape, cfg1.ranks, 5, A0, B0, momentum=mu)
    lr, lam, M, nb = (0.2, 0.1), (0.01, 0.02), 256, 6
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0, momentum=mu, **precision_args) as g:
        g.batches(lr[0], lr[1], lam[0], lam[1], M, 0, nb)
        ref.epoch(c, v, M, 2, 0, lr[0], lr[1], lam[0], lam[1], 0, 0, nb)
        Ag, Bg, _, _ = g.get_params()
    for n in range(3):
        assert float(np.abs(Ag[n] - ref.A[n]).max()) <= 1e-5 * float(np.abs(ref.A[n]).max())
        assert float(np.abs(Bg[n] - ref.B[n]).max()) <= 1e-5 * float(np.abs(ref.B[n]).max())


def test_momentum_epoch_rmse_parity(B, synth, cfg1):
    c, v = cfg1.tensor.split("train")
    tc, tv = cfg1.tensor.split("test")
    A0, B0 = synth.init_params(cfg1.tensor.shape, cfg1.ranks, 5, mode="normal", seed=1)
    mu, lr = 0.8, 0.1
    ref = O.Model(cfg1.tensor.shape, cfg1.ranks, 5, A0, B0, momentum=mu)
    worst = 0.0
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0, momentum=mu) as g:
        for ep in range(4):
            g.epoch(lr, lr, cfg1.lam, cfg1.lam, cfg1.minibatch)
            ref.epoch(c, v, cfg1.minibatch, 2, ep, lr, lr, cfg1.lam, cfg1.lam)
            r_g, m_g = g.rmse(tc, tv)
            r_o, m_o = ref.rmse_mae(tc, tv)
            worst = max(worst, abs(r_g - r_o), abs(m_g - m_o))
    assert worst <= 1e-3, worst


# ---------------------------------------------------------------------------
# Epochs: per-epoch train/test RMSE within 1e-3 absolute over 10 epochs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lr", [1e-3, 0.5])
def test_epoch_rmse_parity_config1(B, synth, cfg1, lr):
    c, v = cfg1.tensor.split("train")
    tc, tv = cfg1.tensor.split("test")
    A0, B0 = synth.init_params(cfg1.tensor.shape, cfg1.ranks, 5, mode="normal", seed=1)
    ref = O.Model(cfg1.tensor.shape, cfg1.ranks, 5, A0, B0)
    worst = 0.0
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0) as g:
        for ep in range(cfg1.epochs):
            g.epoch(lr, lr, cfg1.lam, cfg1.lam, cfg1.minibatch)
            ref.epoch(c, v, cfg1.minibatch, 2, ep, lr, lr, cfg1.lam, cfg1.lam)
            for cc, vv in ((c, v), (tc, tv)):
                r_g, m_g = g.rmse(cc, vv)
                r_o, m_o = ref.rmse_mae(cc, vv)
                worst = max(worst, abs(r_g - r_o), abs(m_g - m_o))
    assert worst <= 1e-3, worst


def test_epochs_are_deterministic(B, synth, cfg1):
    c, v = cfg1.tensor.split("train")
    A0, B0 = synth.init_params(cfg1.tensor.shape, cfg1.ranks, 5, mode="normal", seed=1)
    outs = []
    for _ in range(2):
        with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0) as g:
            for ep in range(2):
                g.epoch(0.5, 0.5, 1e-3, 1e-3, 256)
            outs.append(g.get_params())
    for x, y in zip(outs[0][0] + outs[0][1], outs[1][0] + outs[1][1]):
        assert np.array_equal(x, y)


def test_checkpoint_resume_is_bit_identical(B, synth, cfg1):
    c, v = cfg1.tensor.split("train")
    A0, B0 = synth.init_params(cfg1.tensor.shape, cfg1.ranks, 5, mode="normal", seed=1)
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0) as g:
        for _ in range(3):
            g.epoch(0.5, 0.5, 1e-3, 1e-3, 256)
        full = g.get_params()
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0) as g:
        g.epoch(0.5, 0.5, 1e-3, 1e-3, 256)
        A1, B1, _, ep = g.get_params()
    assert ep == 1
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v) as g:
        g.set_params(A1, B1, epoch=ep)
        g.epoch(0.5, 0.5, 1e-3, 1e-3, 256)
        g.epoch(0.5, 0.5, 1e-3, 1e-3, 256)
        resumed = g.get_params()
    for x, y in zip(full[0] + full[1], resumed[0] + resumed[1]):
        assert np.array_equal(x, y)
    assert resumed[3] == 3


# ---------------------------------------------------------------------------
# BF16 form: BF16 factor mirrors for the gathers, BF16 unfolded core and
# Kronecker rows on tensor cores, FP32 accumulation and FP32 masters.  Bar:
# its train/test RMSE tracks the FP32 form within 1e-3 absolute per epoch.
# ---------------------------------------------------------------------------

def _rmse_track(B, synth, tensor, ranks, R, M, lr, lam, epochs, init="normal"):
    c, v = tensor.split("train")
    tc, tv = tensor.split("test")
    A0, B0 = synth.init_params(tensor.shape, ranks, R, mode=init, seed=1, mean_value=float(np.mean(v)))
    worst = 0.0
    with _gpu(B, tensor.shape, ranks, R, c, v, A0, B0) as g32, \
            _gpu(B, tensor.shape, ranks, R, c, v, A0, B0, precision=1) as g16:
        for ep in range(epochs):
            g32.epoch(lr, lr, lam, lam, M)
            g16.epoch(lr, lr, lam, lam, M)
            for cc, vv in ((c, v), (tc, tv)):
                if cc.shape[0] == 0:
                    continue
                r32, m32 = g32.rmse(cc, vv)
                r16, m16 = g16.rmse(cc, vv)
                worst = max(worst, abs(r32 - r16), abs(m32 - m16))
    return worst


def test_bf16_rmse_tracks_fp32_config1(B, synth, cfg1):
    worst = _rmse_track(B, synth, cfg1.tensor, cfg1.ranks, 5, 256, 0.5, 1e-3, 10)
    assert worst <= 1e-3, worst


def test_bf16_rmse_tracks_fp32_rating(B, synth):
    w = synth.config2(scale=0.004)
    worst = _rmse_track(B, synth, w.tensor, w.ranks, 5, 4096, 0.05, 1e-3, 5, init="rating")
    assert worst <= 1e-3, worst


def test_bf16_rmse_tracks_fp32_4order(B, synth):
    w = synth.config3(scale=0.004)
    worst = _rmse_track(B, synth, w.tensor, w.ranks, 5, 8192, 0.5, 1e-3, 5)
    assert worst <= 1e-3, worst


def test_bf16_step_gradients_close_to_oracle(B, synth, cfg1):
    """One step in the BF16 form: gradients within the BF16 rounding bound
    (2^-8 relative per operand; 2e-2 norm-wise) of the FP64 oracle."""
    c, v = cfg1.tensor.split("train")
    A0, B0 = synth.init_params(cfg1.tensor.shape, cfg1.ranks, 5, mode="normal", seed=1)
    ref = O.Model(cfg1.tensor.shape, cfg1.ranks, 5, A0, B0)
    with _gpu(B, cfg1.tensor.shape, cfg1.ranks, 5, c, v, A0, B0, precision=1) as g:
        pr = g.batches(0.3, 0.2, 0.01, 0.02, 256, 0, 1, probe=True)
    sched = O.perm_range(c.shape[0], 2, 0, 0, 256)
    V, F, nseg = ref.step(c[sched], v[sched], 0.3, 0.2, 0.01, 0.02, probe=True)
    for n in range(3):
        assert _rel(pr["core_V"][n, :5, :5], V[n, :5, :5]) <= 2e-2
        U = int(nseg[n])
        assert pr["nseg"][n] == U
        assert _rel(pr["factor_F"][n, :U, :5], F[n, :U, :5]) <= 2e-2


def test_watchdog_expires_without_fault_and_device_stays_usable(B, cfg1):
    """A bounded wait on a word nothing writes ends with STD_ETIMEOUT after
    its budget (no trap, no hang); a normal epoch runs afterwards."""
    import time
    t0 = time.time()
    assert B.std_watchdog_probe(2_000_000) == B.STD_ETIMEOUT      # 2 ms budget
    assert time.time() - t0 < 5.0
    with pytest.raises(B.StdError):
        B.std_watchdog_probe(10)                                   # budget outside [1e3, 1e10]
    t = cfg1.tensor
    c, v = t.split("train")
    g = B.Tucker(t.shape, cfg1.ranks, c, v, r_core=cfg1.r_core)
    try:
        st = g.epoch(cfg1.lr, cfg1.lr, cfg1.lam, cfg1.lam, cfg1.minibatch)
        assert st["nnz"] == c.shape[0]
    finally:
        g.close()


# ---------------------------------------------------------------------------
# Full size: the Netflix-shaped 100M-nonzero workload in the bench's launch
# configuration (152 CTAs, M = 4096), checked on sampled minibatches the
# oracle computes one by one
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def full2(synth):
    return synth.config2(scale=1.0)


def test_fullsize_schedule_bitexact_sampled_minibatches(B, full2):
    t = full2.tensor
    c, v = t.split("train")
    M = full2.minibatch
    nb = (c.shape[0] + M - 1) // M
    assert c.shape[0] % M != 0          # the last minibatch is ragged
    with B.Tucker(t.shape, full2.ranks, c, v, r_core=full2.r_core) as g:
        for b in (0, nb // 2, nb - 1):
            _check_schedule(B, g, c, M, (b, b + 1))


def test_fullsize_step_gradients_first_minibatch(B, synth, full2):
    _step_case(B, synth, full2.tensor, full2.ranks, full2.r_core, full2.minibatch, batch=0, init="rating",
               lr=(0.05, 0.05))


# ---------------------------------------------------------------------------
# The bench's launch shape over many minibatches: M = 4096 on the rating
# tensor's distributions (Zipf-hot rows that span many chunks) runs on
# min(256, SMs) = 152 CTAs of a GB300 by the library's default choice, the
# full-warp reduce-scatter branch; M = 8192 on the 4-order workload likewise.
# Tag sequencing across minibatches and epochs, the grid barrier and run
# pieces carried over many minibatches are all exercised here.
# ---------------------------------------------------------------------------

def _epoch_parity(B, synth, w, epochs, lr, check_after, bf16=False, lam=1e-3):
    t = w.tensor
    c, v = t.split("train")
    tc, tv = t.split("test")
    R, M = w.r_core, w.minibatch
    A0, B0 = synth.init_params(t.shape, w.ranks, R, mode="rating" if t.meta["rating"] else "normal", seed=1,
                               mean_value=float(np.mean(v)))
    ref = O.Model(t.shape, w.ranks, R, A0, B0)
    worst = {"fp32": 0.0, "bf16": 0.0}
    forms = [("fp32", {})] + ([("bf16", {"precision": 1})] if bf16 else [])
    ctxs = {name: _gpu(B, t.shape, w.ranks, R, c, v, A0, B0, **o) for name, o in forms}
    try:
        for ep in range(epochs):
            ref.epoch(c, v, M, 2, ep, lr, lr, lam, lam)
            for name, g in ctxs.items():
                g.epoch(lr, lr, lam, lam, M)
            if ep + 1 not in check_after:
                continue
            for cc, vv in ((c, v), (tc, tv)):
                r_o, m_o = ref.rmse_mae(cc, vv)
                for name, g in ctxs.items():
                    r_g, m_g = g.rmse(cc, vv)
                    worst[name] = max(worst[name], abs(r_g - r_o), abs(m_g - m_o))
    finally:
        for g in ctxs.values():
            g.close()
    return worst, ref


def test_epoch_rmse_parity_bench_shape_rating_10_epochs(B, synth):
    w = synth.config2(scale=0.004)          # 396k training nonzeros, 97 minibatches of 4096 per epoch
    tc, tv = w.tensor.split("test")
    c, v = w.tensor.split("train")
    A0, B0 = synth.init_params(w.tensor.shape, w.ranks, w.r_core, mode="rating", seed=1,
                               mean_value=float(np.mean(v)))
    start = O.Model(w.tensor.shape, w.ranks, w.r_core, A0, B0)
    start.build_core()
    worst, ref = _epoch_parity(B, synth, w, 10, 0.05, set(range(1, 11)), bf16=True)
    assert worst["fp32"] <= 1e-3, worst
    # the BF16 form against the FP64 oracle, same bar
    assert worst["bf16"] <= 1e-3, worst
    # the run trains: the test RMSE falls by more than the parity bar many times over
    assert ref.rmse_mae(tc, tv)[0] < start.rmse_mae(tc, tv)[0] - 0.02


def test_epoch_rmse_parity_bench_shape_4order(B, synth):
    w = synth.config3(scale=0.004)          # 180k training nonzeros, 22 minibatches of 8192 per epoch
    worst, _ = _epoch_parity(B, synth, w, 5, 0.5, {2, 5}, bf16=True)
    assert worst["fp32"] <= 1e-3, worst
    assert worst["bf16"] <= 1e-3, worst


def test_params_after_8_minibatches_bench_shape(B, synth):
    """Eight consecutive minibatches of 4096 at 152 CTAs from one state:
    every factor and Kruskal matrix within the FP32 step tolerance (1e-5 of
    the parameter scale) of the oracle after the same eight minibatches."""
    w = synth.config2(scale=0.004)
    t = w.tensor
    c, v = t.split("train")
    A0, B0 = synth.init_params(t.shape, w.ranks, w.r_core, mode="rating", seed=1, mean_value=float(np.mean(v)))
    ref = O.Model(t.shape, w.ranks, w.r_core, A0, B0)
    lr, lam = (0.05, 0.05), (1e-3, 1e-3)
    with _gpu(B, t.shape, w.ranks, w.r_core, c, v, A0, B0) as g:
        g.batches(lr[0], lr[1], lam[0], lam[1], 4096, 0, 8)
        Ag, Bg, core, _ = g.get_params()
    ref.epoch(c, v, 4096, 2, 0, lr[0], lr[1], lam[0], lam[1], 0, 0, 8)
    for n in range(3):
        assert float(np.abs(Ag[n] - ref.A[n]).max()) <= 1e-5 * float(np.abs(ref.A[n]).max())
        assert float(np.abs(Bg[n] - ref.B[n]).max()) <= 1e-5 * float(np.abs(ref.B[n]).max())
        # rows the eight minibatches never touched are bit-for-bit the start
        touched = np.zeros(t.shape[n], bool)
        ids = O.perm_range(c.shape[0], 2, 0, 0, 8 * 4096)
        touched[c[ids, n]] = True
        assert np.array_equal(Ag[n][~touched], A0[n][~touched])


@pytest.mark.parametrize("precision,M", [(0, 4096), (1, 4096), (0, 256)])
def test_default_option_kernels_equal_general_kernels(B, synth, precision, M):
    """With the default options the launchers run update kernels compiled
    without the momentum, probe and row-count-normaliser branches; a probe on
    the first minibatch makes the same launch take the general kernel.  Both
    must leave the same bits (152 CTAs at M = 4096; a 16-CTA cluster at 256)."""
    w = synth.config2(scale=0.004)
    t = w.tensor
    c, v = t.split("train")
    A0, B0 = synth.init_params(t.shape, w.ranks, w.r_core, mode="rating", seed=1, mean_value=float(np.mean(v)))
    out = []
    for probe in (False, True):
        with _gpu(B, t.shape, w.ranks, w.r_core, c, v, A0, B0, precision=precision) as g:
            g.batches(0.05, 0.05, 1e-3, 1e-3, M, 0, 6, probe=probe)
            Ag, Bg, core, _ = g.get_params()
            out.append(list(Ag) + list(Bg) + [core])
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("tile", [1, 2, 4])
def test_contraction_tile_gives_the_same_bits(B, synth, tile):
    """std_options.tile forces the FP32 contraction's samples per thread; each
    sample's sums keep one order whatever the tile, so six minibatches of
    4096 on 152 CTAs (27-sample chunks, where the library picks 2) and of 256
    on 16 CTAs leave the same bits as the library's own choice."""
    w = synth.config2(scale=0.004)
    t = w.tensor
    c, v = t.split("train")
    A0, B0 = synth.init_params(t.shape, w.ranks, w.r_core, mode="rating", seed=1, mean_value=float(np.mean(v)))
    for M in (4096, 256):
        out = []
        for tl in (0, tile):
            with _gpu(B, t.shape, w.ranks, w.r_core, c, v, A0, B0, tile=tl) as g:
                g.batches(0.05, 0.05, 1e-3, 1e-3, M, 0, 6)
                Ag, Bg, core, _ = g.get_params()
                out.append(list(Ag) + list(Bg) + [core])
        for x, y in zip(out[0], out[1]):
            assert np.array_equal(x, y)


# ---------------------------------------------------------------------------
# The library's declared limits: order STD_MAX_ORDER = 6, rank and R_core
# STD_MAX_RANK = 32, core size STD_MAX_CORE = 16,384 entries.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,ranks,R,M,nnz", [
    ((9, 8, 7, 6, 5, 4), (2, 3, 2, 2, 3, 2), 3, 64, 1500),     # N = 6
    ((120, 40, 30), (32, 4, 4), 5, 256, 3000),                # J_1 = 32
    ((60, 50, 40), (4, 4, 4), 32, 256, 3000),                 # R_core = 32
    ((100, 90, 40), (32, 32, 16), 2, 128, 600),               # prod J = 16,384
])
def test_step_gradients_at_declared_limits(B, synth, shape, ranks, R, M, nnz):
    t = synth.make_tensor(shape, nnz, [("uniform",)] * len(shape), tuple(min(j, 4) for j in ranks), 0.1, 0.0,
                          seed=37)
    _step_case(B, synth, t, ranks, R, M, batch=0)


def test_epoch_spanning_schedule_segments(B, synth):
    """An epoch longer than one schedule segment (2^22 positions: 1,024
    minibatches of 4096) is scheduled and run segment after segment.  The
    result does not depend on where the segments fall: the epoch equals, bit
    for bit, the same minibatches run as two calls split elsewhere (each call
    starts its own segments), and the schedule of any stretch equals the
    oracle's sampler and tiler."""
    w = synth.config2(scale=0.05)           # 4.95M training nonzeros: 1,209 minibatches, two segments
    t = w.tensor
    c, v = t.split("train")
    nb = (c.shape[0] + 4095) // 4096
    assert c.shape[0] > (1 << 22)
    A0, B0 = synth.init_params(t.shape, w.ranks, w.r_core, mode="rating", seed=1, mean_value=float(np.mean(v)))
    with _gpu(B, t.shape, w.ranks, w.r_core, c, v, A0, B0) as g1, _gpu(B, t.shape, w.ranks, w.r_core, c, v, A0, B0) as g2:
        st = g1.epoch(w.lr, w.lr, w.lam, w.lam, 4096)
        assert st["batches"] == nb
        g2.batches(w.lr, w.lr, w.lam, w.lam, 4096, 0, 300)
        g2.batches(w.lr, w.lr, w.lam, w.lam, 4096, 300, nb)
        P1, P2 = g1.get_params(), g2.get_params()
        for x, y in zip(P1[0] + P1[1], P2[0] + P2[1]):
            assert np.array_equal(x, y)
        # minibatches on both sides of the first segment boundary
        _check_schedule(B, g1, c, 4096, (1022, 1026), epoch=1)


def test_epoch_holds_one_schedule_segment(B, synth):
    """std_sgd_epoch keeps one segment's schedule (2^22 positions) on the
    device; a batched-launch reservation needs the whole epoch's."""
    w = synth.config2(scale=0.05)           # 4.95M training nonzeros: 1,209 minibatches, two segments
    t = w.tensor
    c, v = t.split("train")
    with B.Tucker(t.shape, w.ranks, c, v, r_core=w.r_core) as g:
        g.epoch(w.lr, w.lr, w.lam, w.lam, 4096)
        held = g.device_bytes()
        g.reserve(4096, 16)
        whole = g.device_bytes()
    nb = (c.shape[0] + 4095) // 4096
    words = 24                                          # schedule words per position of a 3-order tensor
    assert whole - held == (nb - 1024) * 4096 * words * 4, (held, whole)
