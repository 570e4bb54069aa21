"""Serving loop on the device: each job's result is the same alone and in the mix.

Jobs of different orders, ranks and sizes arrive while others are being
trained, wait for memory under a budget that holds only some of them, and
advance a few minibatches per tick inside shared persistent launches.  Each
finished model must equal, bit for bit, the model that std_sgd_epoch gives
the same job alone with the same number of CTAs (the batched kernel runs
each tensor's minibatches exactly as the single-tensor kernel does, and a
step boundary only stores and reloads the FP32 parameters); the answers to
queries must equal std_predict on that model; and one job is compared with
the FP64 oracle (test RMSE within 1e-3).
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

# (shape, nnz, ranks, R, dists, minibatch)
JOBS = [
    ((300, 200, 100), 20000, (8, 8, 8), 5, [("zipf", 1.2), ("zipf", 1.2), ("uniform",)], 256),
    ((80, 70, 60, 12), 9000, (4, 4, 4, 4), 3, [("uniform",)] * 4, 256),
    ((120, 90, 60), 6000, (4, 4, 4), 4, [("uniform",)] * 3, 256),
    ((500, 40, 30), 3000, (16, 16, 16), 5, [("uniform",)] * 3, 256),
    ((200, 150, 90), 12000, (8, 4, 16), 5, [("zipf", 1.1), ("uniform",), ("uniform",)], 256),
]
LR, LAM, EPOCHS, GROUP = 0.1, 1e-3, 2, 4


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def tensors():
    from paper_2012_03550_gb300 import synth as s
    return [s.make_tensor(shape, nnz, dists, ranks, 0.05, 0.1, seed=300 + k)
            for k, (shape, nnz, ranks, R, dists, M) in enumerate(JOBS)]


def _job(serve, k, t, **kw):
    shape, nnz, ranks, R, dists, M = JOBS[k]
    c, v = t.split("train")
    return serve.Job(shape=shape, ranks=ranks, coords=c, values=v, epochs=EPOCHS, minibatch=M,
                     lr_a=LR, lr_b=LR, lam_a=LAM, lam_b=LAM, r_core=R,
                     options={"seed_init": 11 + k, "seed_sched": 5 + k}, fetch_params=True, **kw)


def _alone(B, k, t, precision, ctas=GROUP):
    shape, nnz, ranks, R, dists, M = JOBS[k]
    c, v = t.split("train")
    g = B.Tucker(shape, ranks, c, v, r_core=R, ctas=ctas, precision=precision, seed_init=11 + k,
                 seed_sched=5 + k)
    for _ in range(EPOCHS):
        g.epoch(LR, LR, LAM, LAM, M)
    return g


def _by_size(job):
    # a job's group size from its own shape only
    return 8 if job.nnz >= 10000 else 2


@pytest.mark.parametrize("precision,policy", [(0, None), (1, None), (0, _by_size)])
def test_each_job_is_the_same_alone_and_in_the_mix(B, tensors, precision, policy):
    from paper_2012_03550_gb300 import serve
    eng = serve.CudaEngine(precision=precision, max_query=512)
    # footprints with the reservation the server makes, to size a budget that holds two or three jobs
    sizes = []
    for k, t in enumerate(tensors):
        h = eng.open(_job(serve, k, t), 1 << 40, GROUP)
        sizes.append(eng.device_bytes(h))
        eng.close(h)
    budget = sorted(sizes)[-1] + sorted(sizes)[-2] + min(sizes) // 2
    srv = serve.Server(eng, budget_bytes=budget, batches_per_tick=7, ctas_per_tensor=policy or GROUP)
    rng = np.random.default_rng(0)
    queries = []
    try:
        ids = [srv.submit(_job(serve, 0, tensors[0])), srv.submit(_job(serve, 1, tensors[1]))]
        srv.tick()
        srv.tick()
        ids.append(srv.submit(_job(serve, 2, tensors[2])))
        srv.tick()
        ids += [srv.submit(_job(serve, 3, tensors[3])), srv.submit(_job(serve, 4, tensors[4]))]
        peak = 0
        waited = False
        while not srv.idle():
            srv.tick()
            peak = max(peak, srv.used_bytes())
            waited = waited or len(srv.queue) > 0
            assert srv.used_bytes() <= budget
            for j in list(srv.running):
                if j.status == "running" and rng.random() < 0.2:
                    k = int(rng.integers(1, 700))
                    crd = np.stack([rng.integers(0, s, size=k) for s in j.shape], axis=1).astype(np.int32)
                    queries.append(srv.query(j.id, crd))
        assert waited, "the budget should have made some job wait"
        # final queries against every finished job that is still resident
        finals = {}
        for jid in ids:
            j = srv.jobs[jid]
            if j.handle is not None:
                crd = np.stack([rng.integers(0, s, size=300) for s in j.shape], axis=1).astype(np.int32)
                finals[jid] = srv.query(jid, crd)
        srv.tick()
        for k, jid in enumerate(ids):
            j = srv.jobs[jid]
            assert j.status in ("done", "evicted"), (jid, j.status, j.error)
            assert len(j.epoch_times) == EPOCHS
            assert j.ctas == (policy(j) if policy else GROUP)
            g = _alone(B, k, tensors[k], precision, j.ctas)
            A, Bm, core, ep = g.get_params()
            A2, B2, core2, ep2 = j.params
            assert ep == ep2 == EPOCHS
            assert all(np.array_equal(x, y) for x, y in zip(A, A2)), f"job {k}: factors differ"
            assert all(np.array_equal(x, y) for x, y in zip(Bm, B2)), f"job {k}: Kruskal columns differ"
            assert np.array_equal(core, core2)
            if jid in finals:
                q = finals[jid]
                assert not q.error and np.array_equal(q.values, g.predict(q.coords))
            g.close()
        assert all(not q.error and q.values is not None and q.values.shape[0] == q.coords.shape[0]
                   for q in queries)
        r = srv.report()
        assert r["jobs_done"] == len(JOBS) and r["query_p99_s"] is not None
    finally:
        srv.shutdown()


def test_served_job_tracks_oracle(B, tensors):
    from paper_2012_03550_gb300 import serve
    k = 2
    t = tensors[k]
    shape, nnz, ranks, R, dists, M = JOBS[k]
    c, v = t.split("train")
    tc, tv = t.split("test")
    # the initial model the job draws on the device (same seed, epoch 0)
    g0 = B.Tucker(shape, ranks, c, v, r_core=R, seed_init=11 + k, seed_sched=5 + k)
    A0, B0, _, _ = g0.get_params()
    g0.close()
    eng = serve.CudaEngine(precision=0)
    srv = serve.Server(eng, budget_bytes=1 << 34, batches_per_tick=5, ctas_per_tensor=GROUP)
    try:
        jid = srv.submit(_job(serve, k, t))
        srv.run_until_idle()
        A, Bm, _, _ = srv.jobs[jid].params
    finally:
        srv.shutdown()
    ref = O.Model(shape, ranks, R, A0, B0)
    for ep in range(EPOCHS):
        ref.epoch(c, v, M, 5 + k, ep, LR, LR, LAM, LAM)
    got = O.Model(shape, ranks, R, A, Bm)
    got.build_core()
    r_g, m_g = got.rmse_mae(tc, tv)
    r_o, m_o = ref.rmse_mae(tc, tv)
    assert abs(r_g - r_o) <= 1e-3 and abs(m_g - m_o) <= 1e-3, (r_g, r_o, m_g, m_o)


def test_epoch_in_progress_is_protected(B, tensors):
    shape, nnz, ranks, R, dists, M = JOBS[2]
    c, v = tensors[2].split("train")
    g = B.Tucker(shape, ranks, c, v, r_core=R)
    try:
        with B.Batch([g], ctas_per_tensor=2) as bt:
            st = bt.step(LR, LR, LAM, LAM, M, 3)
            assert st["nnz"] == 3 * M and st["graph_replayed"] == 0
            assert g.progress() == (0, 3)
            with pytest.raises(B.StdError):
                g.epoch(LR, LR, LAM, LAM, M)           # std_sgd_epoch refuses a context mid-epoch
            with pytest.raises(B.StdError):
                bt.step(LR, LR, LAM, LAM, M // 2, 1)   # and a step with another minibatch size
            st = bt.step(LR, LR, LAM, LAM, M, 10 ** 6)
            assert st["nnz"] == c.shape[0] - 3 * M
            assert st["graph_replayed"] == 1        # same tensors and group size: the captured graph
            assert g.progress() == (1, 0)
        g.epoch(LR, LR, LAM, LAM, M)
        assert g.progress() == (2, 0)
    finally:
        g.close()


def test_predict_many_equals_each_context_alone(B, tensors):
    """One launch over jobs of orders 3 and 4 gives each job's std_predict bit for bit."""
    rng = np.random.default_rng(3)
    gs, crds = [], []
    try:
        for k in (0, 1, 3):
            shape, nnz, ranks, R, dists, M = JOBS[k]
            c, v = tensors[k].split("train")
            g = B.Tucker(shape, ranks, c, v, r_core=R, seed_init=40 + k)
            g.epoch(LR, LR, LAM, LAM, M)
            gs.append(g)
            n = (1, 700, 4096)[k % 3]
            crds.append(np.stack([rng.integers(0, s, size=n) for s in shape], axis=1).astype(np.int32))
        outs = B.predict_many(gs, crds)
        for g, cc, o in zip(gs, crds, outs):
            assert np.array_equal(o, g.predict(cc))
        bad = crds[1].copy()
        bad[5, 0] = gs[1].shape[0]
        with pytest.raises(B.StdError):
            B.predict_many(gs, [crds[0], bad, crds[2]])
    finally:
        for g in gs:
            g.close()
