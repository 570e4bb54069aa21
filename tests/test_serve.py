"""Host logic of the serving loop, against a fake engine (no device).

The fake engine mirrors the library's contract for batched steps: a context
keeps its position in the epoch, a step advances each tensor by up to K
minibatches, a tensor that completes its epoch advances its counter; its
memory footprint is fixed when it is opened, and opening fails when the
footprint exceeds the memory offered.
"""
import numpy as np
import pytest

from paper_2012_03550_gb300.serve import BudgetExceeded, Job, Server


class FakeHandle:
    def __init__(self, job, bytes_):
        self.job = job
        self.bytes = bytes_
        self.epoch = 0
        self.cursor = 0
        self.closed = False


class FakeEngine:
    max_query = 1000

    def __init__(self, bytes_per_nnz=10, tuned_group=4):
        self.bytes_per_nnz = bytes_per_nnz
        self.tuned_group = tuned_group
        self.open_handles = []
        self.steps = []           # (ids, key, K, G)
        self.predicts = []        # (job id, k)

    def footprint(self, job):
        return job.nnz * self.bytes_per_nnz

    def open(self, job, budget_bytes, ctas_per_tensor):
        assert ctas_per_tensor >= 1
        if self.footprint(job) > budget_bytes:
            raise BudgetExceeded("over budget")
        h = FakeHandle(job, self.footprint(job))
        self.open_handles.append(h)
        return h

    def device_bytes(self, h):
        return h.bytes

    def close(self, h):
        assert not h.closed
        h.closed = True
        self.open_handles.remove(h)

    def step(self, handles, key, K, sizes):
        assert all(not h.closed for h in handles)
        assert len(sizes) == len(handles)
        g = sizes[0] if sizes[0] > 0 else self.tuned_group
        self.steps.append((tuple(h.job.id for h in handles), key, K, tuple(sizes)))
        nnz = 0
        M = key[4]
        for h in handles:
            nb = -(-h.job.nnz // M)
            e1 = min(nb, h.cursor + K)
            nnz += min(e1 * M, h.job.nnz) - h.cursor * M
            h.cursor = e1
            if h.cursor >= nb:
                h.cursor = 0
                h.epoch += 1
        return {"seconds": 1e-3, "update_seconds": 1e-3, "nnz": nnz, "nnz_per_s": nnz / 1e-3,
                "tensors": len(handles), "ctas_per_tensor": g}

    def progress(self, h):
        return h.epoch, h.cursor

    def predict(self, h, coords):
        assert not h.closed and coords.shape[0] <= self.max_query
        self.predicts.append((h.job.id, coords.shape[0]))
        return coords.sum(axis=1).astype(np.float32) + 1000.0 * h.job.id

    def params(self, h):
        return ("params", h.job.id, h.epoch)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


def job(nnz, epochs=1, M=100, order=3, **kw):
    coords = np.zeros((nnz, order), np.int32)
    return Job(shape=(10,) * order, ranks=(4,) * order, coords=coords, values=np.zeros(nnz, np.float32),
               epochs=epochs, minibatch=M, **kw)


def test_budget_is_never_exceeded_and_jobs_wait_in_order():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=25_000, batches_per_tick=3, clock=Clock(), keep_finished=False)
    ids = [srv.submit(job(n, epochs=1)) for n in (1000, 1200, 800, 2000, 300)]
    admitted_order = []
    while not srv.idle():
        srv.tick()
        assert srv.used_bytes() <= srv.budget
        assert sum(h.bytes for h in eng.open_handles) <= srv.budget
        for j in srv.running:
            if j.id not in admitted_order:
                admitted_order.append(j.id)
    # head of line: admission order equals arrival order
    assert admitted_order == sorted(admitted_order)
    assert all(srv.jobs[i].status == "released" for i in ids)
    assert not eng.open_handles


def test_epoch_accounting_and_tick_count():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=10**9, batches_per_tick=4, clock=Clock())
    j = srv.submit(job(1050, epochs=3, M=100))      # 11 minibatches per epoch -> 3 steps per epoch
    srv.run_until_idle()
    J = srv.jobs[j]
    assert len(J.epoch_times) == 3 and J.status == "done"
    assert srv.ticks == 9
    assert srv.nnz == 3 * 1050
    assert all(lat > 0 for lat in J.epoch_latencies())


def test_group_size_fixed_after_first_tuned_step():
    eng = FakeEngine(tuned_group=8)
    srv = Server(eng, budget_bytes=10**9, batches_per_tick=2, clock=Clock())
    srv.submit(job(500))
    srv.tick()
    srv.submit(job(500))
    srv.run_until_idle()
    assert eng.steps[0][3] == (0,)                 # the first step asks the tuner
    assert all(set(s[3]) == {8} for s in eng.steps[1:])   # later steps reuse its choice


def test_per_job_group_sizes_from_a_policy_stay_fixed():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=10**9, batches_per_tick=2, clock=Clock(),
                 ctas_per_tensor=lambda job: 8 if job.nnz >= 1000 else 2)
    a = srv.submit(job(1500))
    b = srv.submit(job(300))
    srv.tick()
    c = srv.submit(job(2000))
    srv.run_until_idle()
    assert srv.jobs[a].ctas == 8 and srv.jobs[b].ctas == 2 and srv.jobs[c].ctas == 8
    for ids, key, K, sizes in eng.steps:
        assert sizes == tuple(srv.jobs[i].ctas for i in ids)


def test_jobs_with_different_hyperparameters_step_in_separate_launches():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=10**9, batches_per_tick=100, clock=Clock(), ctas_per_tensor=2)
    a = srv.submit(job(300, lr_a=0.1))
    b = srv.submit(job(300, lr_a=0.2))
    c = srv.submit(job(300, lr_a=0.1))
    srv.tick()
    launches = {s[0] for s in eng.steps}
    assert launches == {(a, c), (b,)}


def test_finished_models_stay_for_queries_and_are_evicted_oldest_first():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=20_000, batches_per_tick=100, clock=Clock())
    a = srv.submit(job(1000, fetch_params=True))
    b = srv.submit(job(900))
    srv.tick()
    assert srv.jobs[a].status == "done" and srv.jobs[a].params == ("params", a, 1)
    q = srv.query(a, np.array([[1, 2, 3]], np.int32))
    srv.tick()
    assert q.values is not None and q.values[0] == 6.0 + 1000.0 * a
    c = srv.submit(job(1500))                      # needs the room of a (evicted first), then b
    srv.tick()
    assert srv.jobs[a].status == "evicted" and srv.jobs[b].status == "evicted"
    assert srv.jobs[c].status in ("running", "done")
    late = srv.query(a, np.array([[0, 0, 0]], np.int32))
    srv.tick()
    assert late.error and late.values is None


def test_oversized_job_is_rejected_not_deadlocked():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=5_000, clock=Clock())
    big = srv.submit(job(10_000))
    small = srv.submit(job(100))
    srv.run_until_idle()
    assert srv.jobs[big].status == "rejected" and srv.jobs[small].status == "done"


def test_queries_are_batched_per_job_and_split_back():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=10**9, batches_per_tick=1, clock=Clock())
    a = srv.submit(job(1000, epochs=5))
    b = srv.submit(job(1000, epochs=5))
    srv.tick()
    rng = np.random.default_rng(0)
    qs = []
    for k in (1, 7, 700, 600, 3):
        for jid in (a, b):
            qs.append((jid, srv.query(jid, rng.integers(0, 10, size=(k, 3)).astype(np.int32))))
    eng.predicts.clear()
    srv.tick()
    # 1311 coordinates per job in pieces of at most max_query: two launches per job
    assert sorted(eng.predicts) == sorted([(a, 1000), (a, 311), (b, 1000), (b, 311)])
    for jid, q in qs:
        assert np.array_equal(q.values, q.coords.sum(axis=1).astype(np.float32) + 1000.0 * jid)
        assert q.answered >= q.submitted


def test_query_for_a_queued_job_waits_for_admission():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=15_000, batches_per_tick=1, clock=Clock())
    a = srv.submit(job(1000, epochs=2))
    b = srv.submit(job(1000))                       # waits: only one fits
    srv.tick()
    q = srv.query(b, np.array([[1, 1, 1]], np.int32))
    srv.tick()
    assert srv.jobs[b].status == "queued" and q.values is None and not q.error
    srv.run_until_idle()
    assert q.values is not None and not q.error


def test_report_fields():
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=10**9, batches_per_tick=2, clock=Clock())
    for n in (300, 500, 700):
        srv.submit(job(n, epochs=2))
    srv.query(0, np.zeros((4, 3), np.int32))
    srv.run_until_idle()
    r = srv.report()
    assert r["jobs_done"] == 3 and r["queries_answered"] == 1 and r["nnz"] == 2 * 1500
    for k in ("job_epoch_p50_s", "job_epoch_p99_s", "query_p50_s", "query_p99_s", "job_p99_s"):
        assert r[k] is not None and r[k] > 0
    assert r["job_epoch_p50_s"] <= r["job_epoch_p99_s"]


def test_bad_server_arguments():
    with pytest.raises(ValueError):
        Server(FakeEngine(), budget_bytes=0)
    with pytest.raises(ValueError):
        Server(FakeEngine(), budget_bytes=10, batches_per_tick=0)


class FakeManyEngine(FakeEngine):
    def __init__(self):
        super().__init__()
        self.many = []

    def predict_many(self, handles, coords_list):
        self.many.append(tuple((h.job.id, c.shape[0]) for h, c in zip(handles, coords_list)))
        return [c.sum(axis=1).astype(np.float32) + 1000.0 * h.job.id for h, c in zip(handles, coords_list)]


def test_queries_of_all_jobs_go_in_one_launch_when_the_engine_allows():
    eng = FakeManyEngine()
    srv = Server(eng, budget_bytes=10**9, batches_per_tick=1, clock=Clock())
    a = srv.submit(job(1000, epochs=5))
    b = srv.submit(job(1000, epochs=5))
    srv.tick()
    rng = np.random.default_rng(1)
    qs = [(jid, srv.query(jid, rng.integers(0, 10, size=(k, 3)).astype(np.int32)))
          for k in (5, 2000, 3) for jid in (a, b)]
    srv.tick()
    assert eng.many == [((a, 2008), (b, 2008))] and not eng.predicts
    for jid, q in qs:
        assert np.array_equal(q.values, q.coords.sum(axis=1).astype(np.float32) + 1000.0 * jid)


class _FakeBatch:
    log = []

    def __init__(self, members, ctas):
        self.members = list(members)
        self.closed = False
        _FakeBatch.log.append(("create", len(members), ctas))

    def reset(self, members):
        assert not self.closed
        self.members = list(members)
        _FakeBatch.log.append(("reset", len(members)))

    def set_groups(self, sizes):
        assert len(sizes) == len(self.members)
        _FakeBatch.log.append(("groups", tuple(sizes)))

    def step(self, *args):
        assert not self.closed
        return {"seconds": 0.0, "nnz": 0, "ctas_per_tensor": 4}

    def close(self):
        self.closed = True
        _FakeBatch.log.append(("close",))


class _FakeBinding:
    Batch = _FakeBatch


class _H:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def test_engine_keeps_one_batch_per_key_and_forgets_closed_jobs():
    from paper_2012_03550_gb300.serve import CudaEngine
    eng = CudaEngine.__new__(CudaEngine)
    eng._b = _FakeBinding
    eng._batches = {}
    _FakeBatch.log = []
    key = (0.1, 0.1, 0.0, 0.0, 256)
    a, b, c = _H(), _H(), _H()
    eng.step([a, b], key, 4, [4, 8])
    eng.step([a, b], key, 4, [4, 8])            # same jobs and sizes: nothing re-pointed
    eng.step([a, b, c], key, 4, [4, 8, 4])      # a job joins: reset + sizes
    eng.close(b)                                # a member goes: the batch forgets it first
    eng.close(a)
    eng.step([c], key, 4, [4])
    eng.close(c)                                # the last member: the batch is closed
    assert _FakeBatch.log == [("create", 2, 4), ("groups", (4, 8)),
                              ("reset", 3), ("groups", (4, 8, 4)),
                              ("reset", 2), ("reset", 1),
                              ("groups", (4,)), ("close",)]
    assert a.closed and b.closed and c.closed and not eng._batches
