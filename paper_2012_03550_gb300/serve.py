"""Continuous-batching server for SGD_Tucker decomposition jobs and queries.

A job is one sparse tensor (COO, mode sizes, ranks, options) to decompose for
a number of epochs of Algorithm 1; a query asks a job's model for the values
x-hat at a list of coordinates (Def. 6 with the core of Eq. 4).  The server
works in ticks.  Each tick

1. admits queued jobs in arrival order while the device-memory budget (and the
   optional slot limit) allows.  A job's footprint is exact, not estimated:
   its context is created with the remaining budget as its allocation cap and
   then reserved (std_reserve allocates the epoch schedule, the exchange
   scratch and the query staging up front), so the steps and queries that
   follow allocate nothing.  A job that does not fit waits at the head of the
   queue; finished models that are still resident are evicted oldest first to
   make room; a job larger than the whole budget is rejected;
2. answers every pending query in one launch over all jobs
   (std_predict_many, each job's queries concatenated), or one std_predict
   per job when the engine has no multi-job form;
3. advances every admitted job by up to `batches_per_tick` minibatches of its
   current epoch with one std_batch_step per group of jobs that share
   hyperparameters: all jobs of a group run in the same persistent launch,
   each on its own CTA group, each exactly as it would run alone;
4. records epoch completions and finishes the jobs that reached their epoch
   count.  A finished job's model stays resident for queries (and may be
   copied to the host) until it is released or evicted.

The server holds no arithmetic of the method: every step runs in the
library's kernels behind the engine object.  The engine is an argument so
that the scheduling logic can be exercised without a device.
Latencies are host wall-clock times (time.perf_counter by default).
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np


class BudgetExceeded(Exception):
    """The engine could not fit a job into the memory it was offered."""


@dataclasses.dataclass
class Job:
    shape: Tuple[int, ...]
    ranks: Tuple[int, ...]
    coords: np.ndarray            # nnz x N int32
    values: np.ndarray            # nnz float32
    epochs: int = 1
    minibatch: int = 256
    lr_a: float = 1e-3
    lr_b: float = 1e-3
    lam_a: float = 1e-3
    lam_b: float = 1e-3
    r_core: int = 5
    options: Dict[str, object] = dataclasses.field(default_factory=dict)
    fetch_params: bool = False    # copy A, B, core to the host when the job finishes
    # filled in by the server
    id: int = -1
    status: str = "new"           # queued, running, done, evicted, released, rejected
    error: str = ""
    arrival: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    epoch_times: List[float] = dataclasses.field(default_factory=list)
    device_bytes: int = 0
    ctas: int = 0                 # CTAs of the job's group in every launch (0: tuned at the first step)
    params: Optional[tuple] = None
    handle: object = None

    @property
    def nnz(self) -> int:
        return int(self.coords.shape[0])

    def key(self) -> tuple:
        return (float(self.lr_a), float(self.lr_b), float(self.lam_a), float(self.lam_b), int(self.minibatch))

    def epoch_latencies(self) -> List[float]:
        """Wall time of each epoch: admission to the first epoch's end, then epoch end to epoch end."""
        out, t = [], self.admitted
        for e in self.epoch_times:
            out.append(e - t)
            t = e
        return out


@dataclasses.dataclass
class Query:
    job_id: int
    coords: np.ndarray            # k x N int32
    submitted: float = 0.0
    answered: float = 0.0
    values: Optional[np.ndarray] = None
    error: str = ""


class CudaEngine:
    """The library behind the server: one context per job, batched steps."""

    def __init__(self, precision: int = 0, max_query: int = 4096):
        from . import binding
        self._b = binding
        self.precision = int(precision)
        self.max_query = int(max_query)
        self._batches: Dict[tuple, object] = {}   # hyperparameter key -> (members, sizes, Batch)

    def open(self, job: Job, budget_bytes: int, ctas_per_tensor: int):
        b = self._b
        if budget_bytes <= 0:
            raise BudgetExceeded("no device memory left in the budget")
        opts = dict(job.options)
        opts["precision"] = self.precision
        opts["hbm_budget_bytes"] = int(budget_bytes)
        t = None
        try:
            t = b.Tucker(job.shape, job.ranks, job.coords, job.values, r_core=job.r_core, **opts)
            t.reserve(job.minibatch, ctas_per_tensor, self.max_query)
        except b.StdError as e:
            if t is not None:
                t.close()
            if e.code == b.STD_ENOMEM:
                raise BudgetExceeded(str(e)) from None
            raise
        return t

    def device_bytes(self, h) -> int:
        return h.device_bytes()

    def close(self, h) -> None:
        # a batch that still lists this job forgets it before the context goes
        for key in [k for k, v in self._batches.items() if any(m is h for m in v[0])]:
            members, _, bt = self._batches[key]
            rest = [m for m in members if m is not h]
            if rest:
                bt.reset(rest)
                self._batches[key] = (rest, None, bt)   # sizes are set again at the next step
            else:
                self._batches.pop(key)[2].close()
        h.close()

    def step(self, handles: Sequence, key: tuple, batches: int, sizes: Sequence[int]) -> dict:
        """One batched step; sizes[i] = CTAs of handle i's group (all 0: the
        library's tuner picks one size for every tensor).  One batch object
        per hyperparameter key is kept and re-pointed at the current jobs."""
        b = self._b
        sizes = [int(x) for x in sizes]
        tune = all(x == 0 for x in sizes)
        entry = self._batches.get(key)
        if entry is None:
            bt = b.Batch(handles, -1 if tune else min(sizes))   # -1: tuned, one size for all
            changed = True
        else:
            members, old_sizes, bt = entry
            same = len(members) == len(handles) and all(m is h for m, h in zip(members, handles))
            if not same:
                bt.reset(list(handles))
            changed = not same or old_sizes != sizes
        if changed and not tune:
            bt.set_groups(sizes)      # every job at its own size, whatever the others are
        self._batches[key] = (list(handles), sizes, bt)
        lr_a, lr_b, lam_a, lam_b, m = key
        return bt.step(lr_a, lr_b, lam_a, lam_b, m, batches)

    def progress(self, h) -> Tuple[int, int]:
        return h.progress()

    def predict(self, h, coords: np.ndarray) -> np.ndarray:
        return h.predict(coords)

    def predict_many(self, handles: Sequence, coords_list: Sequence[np.ndarray]) -> List[np.ndarray]:
        """Every job's queries in one launch (std_predict_many)."""
        return self._b.predict_many(handles, coords_list)

    def params(self, h):
        return h.get_params()

    def shutdown(self) -> None:
        for _, _, bt in self._batches.values():
            bt.close()
        self._batches.clear()


def _percentile(xs: Sequence[float], q: float) -> Optional[float]:
    if len(xs) == 0:
        return None
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


class Server:
    """Admission, ticks and bookkeeping; see the module docstring."""

    def __init__(self, engine, budget_bytes: int, batches_per_tick: int = 32, max_jobs: int = 0,
                 ctas_per_tensor=0, keep_finished: bool = True,
                 clock: Callable[[], float] = time.perf_counter):
        """ctas_per_tensor: CTAs of every job's group (0: tuned at the first
        step), or a function of the job giving its own size; either way a
        job keeps its size for its whole life, so its result does not depend
        on the jobs it shares launches with."""
        if budget_bytes <= 0:
            raise ValueError("budget_bytes must be positive")
        if batches_per_tick < 1:
            raise ValueError("batches_per_tick must be >= 1")
        self.engine = engine
        self.budget = int(budget_bytes)
        self.batches_per_tick = int(batches_per_tick)
        self.max_jobs = int(max_jobs)
        self.policy = ctas_per_tensor if callable(ctas_per_tensor) else None
        self.group = 0 if self.policy else int(ctas_per_tensor)   # 0: chosen by the tuner at the first step
        self.keep_finished = keep_finished
        self.clock = clock
        self.jobs: Dict[int, Job] = {}
        self.queue: collections.deque = collections.deque()
        self.running: List[Job] = []
        self.resident_done: collections.OrderedDict = collections.OrderedDict()
        self.pending: List[Query] = []
        self.answered: List[Query] = []
        self.ticks = 0
        self.nnz = 0
        self.gpu_seconds = 0.0
        self.step_seconds = 0.0
        self._next_id = 0

    # -- requests ----------------------------------------------------------
    def submit(self, job: Job, now: Optional[float] = None) -> int:
        job.id = self._next_id
        self._next_id += 1
        job.arrival = self.clock() if now is None else now
        job.status = "queued"
        self.jobs[job.id] = job
        self.queue.append(job)
        return job.id

    def query(self, job_id: int, coords, now: Optional[float] = None) -> Query:
        q = Query(job_id=job_id, coords=np.ascontiguousarray(coords, dtype=np.int32))
        q.submitted = self.clock() if now is None else now
        self.pending.append(q)
        return q

    def release(self, job_id: int) -> None:
        """Free a finished job's resident model."""
        j = self.jobs[job_id]
        if j.id in self.resident_done:
            del self.resident_done[j.id]
            self.engine.close(j.handle)
            j.handle = None
            j.status = "released"

    # -- accounting --------------------------------------------------------
    def used_bytes(self) -> int:
        return sum(j.device_bytes for j in self.running) + sum(j.device_bytes for j in self.resident_done.values())

    def idle(self) -> bool:
        return not self.queue and not self.running and not self.pending

    # -- one tick ----------------------------------------------------------
    def _evict_oldest_done(self) -> bool:
        if not self.resident_done:
            return False
        _, j = self.resident_done.popitem(last=False)
        self.engine.close(j.handle)
        j.handle = None
        j.status = "evicted"
        return True

    def _admit(self) -> None:
        while self.queue and (self.max_jobs <= 0 or len(self.running) < self.max_jobs):
            job = self.queue[0]
            job.ctas = int(self.policy(job)) if self.policy else self.group
            free = self.budget - self.used_bytes()
            try:
                h = self.engine.open(job, free, job.ctas if job.ctas > 0 else 32)
            except BudgetExceeded as e:
                if self._evict_oldest_done():
                    continue
                if not self.running:
                    # nothing else holds memory: the job can never fit
                    self.queue.popleft()
                    job.status = "rejected"
                    job.error = str(e)
                    continue
                return
            except Exception as e:  # a job the library refuses (shape, ranks) fails alone
                self.queue.popleft()
                job.status = "rejected"
                job.error = str(e)
                continue
            self.queue.popleft()
            job.handle = h
            job.device_bytes = int(self.engine.device_bytes(h))
            job.admitted = self.clock()
            job.status = "running"
            self.running.append(job)

    def _answer(self) -> None:
        if not self.pending:
            return
        waiting: List[Query] = []
        per_job: Dict[int, List[Query]] = collections.defaultdict(list)
        for q in self.pending:
            j = self.jobs.get(q.job_id)
            if j is None or j.status in ("evicted", "released", "rejected"):
                q.error = "job is not resident" if j is not None else "unknown job"
                q.answered = self.clock()
                self.answered.append(q)
            elif j.handle is None:
                waiting.append(q)           # queued: answered once the job is admitted
            else:
                per_job[q.job_id].append(q)
        jids = list(per_job)
        coords_of = {jid: (np.concatenate([q.coords for q in per_job[jid]], axis=0) if len(per_job[jid]) > 1
                           else per_job[jid][0].coords) for jid in jids}
        vals_of = {}
        if jids and hasattr(self.engine, "predict_many"):
            outs = self.engine.predict_many([self.jobs[jid].handle for jid in jids], [coords_of[jid] for jid in jids])
            vals_of = dict(zip(jids, outs))
        else:
            for jid in jids:
                coords = coords_of[jid]
                limit = getattr(self.engine, "max_query", 0) or coords.shape[0]
                vals = np.empty(coords.shape[0], np.float32)
                for a in range(0, coords.shape[0], limit):
                    vals[a:a + limit] = self.engine.predict(self.jobs[jid].handle, coords[a:a + limit])
                vals_of[jid] = vals
        for jid in jids:
            qs = per_job[jid]
            vals = vals_of[jid]
            t = self.clock()
            off = 0
            for q in qs:
                k = q.coords.shape[0]
                q.values = vals[off:off + k]
                off += k
                q.answered = t
                self.answered.append(q)
        self.pending = waiting

    def _step(self) -> None:
        if not self.running:
            return
        groups: Dict[tuple, List[Job]] = collections.OrderedDict()
        for j in self.running:
            groups.setdefault(j.key(), []).append(j)
        t0 = self.clock()
        for key, js in groups.items():
            st = self.engine.step([j.handle for j in js], key, self.batches_per_tick, [j.ctas for j in js])
            if any(j.ctas == 0 for j in js):
                # the tuner ran: every job keeps the size it chose
                self.group = int(st["ctas_per_tensor"])
                for j in self.running:
                    if j.ctas == 0:
                        j.ctas = self.group
            self.nnz += int(st["nnz"])
            self.gpu_seconds += float(st["seconds"])
        t1 = self.clock()
        self.step_seconds += t1 - t0
        still: List[Job] = []
        for j in self.running:
            epoch, _ = self.engine.progress(j.handle)
            done_epochs = int(epoch) - len(j.epoch_times)
            for _ in range(max(0, done_epochs)):
                j.epoch_times.append(t1)
            if len(j.epoch_times) >= j.epochs:
                j.finished = t1
                j.status = "done"
                if j.fetch_params:
                    j.params = self.engine.params(j.handle)
                if self.keep_finished:
                    self.resident_done[j.id] = j
                else:
                    self.engine.close(j.handle)
                    j.handle = None
                    j.status = "released"
            else:
                still.append(j)
        self.running = still

    def tick(self) -> None:
        self._admit()
        self._answer()
        self._step()
        self.ticks += 1

    def run_until_idle(self, max_ticks: int = 1_000_000) -> None:
        for _ in range(max_ticks):
            if self.idle():
                return
            self.tick()
        raise RuntimeError("server did not drain within max_ticks")

    def shutdown(self) -> None:
        for j in list(self.running) + list(self.resident_done.values()):
            if j.handle is not None:
                self.engine.close(j.handle)
                j.handle = None
        self.running = []
        self.resident_done.clear()
        if hasattr(self.engine, "shutdown"):
            self.engine.shutdown()

    # -- report ------------------------------------------------------------
    def report(self) -> dict:
        done = [j for j in self.jobs.values() if j.finished > 0]
        ep = [x for j in done for x in j.epoch_latencies()]
        job_lat = [j.finished - j.arrival for j in done]
        wait = [j.admitted - j.arrival for j in self.jobs.values() if j.admitted > 0]
        ql = [q.answered - q.submitted for q in self.answered if not q.error]
        return {
            "jobs_submitted": len(self.jobs),
            "jobs_done": len(done),
            "jobs_rejected": sum(1 for j in self.jobs.values() if j.status == "rejected"),
            "queries_answered": sum(1 for q in self.answered if not q.error),
            "queries_failed": sum(1 for q in self.answered if q.error),
            "ticks": self.ticks,
            "nnz": self.nnz,
            "gpu_seconds": self.gpu_seconds,
            "step_seconds": self.step_seconds,
            "job_epoch_p50_s": _percentile(ep, 50), "job_epoch_p99_s": _percentile(ep, 99),
            "job_p50_s": _percentile(job_lat, 50), "job_p99_s": _percentile(job_lat, 99),
            "queue_wait_p50_s": _percentile(wait, 50), "queue_wait_p99_s": _percentile(wait, 99),
            "query_p50_s": _percentile(ql, 50), "query_p99_s": _percentile(ql, 99),
        }
