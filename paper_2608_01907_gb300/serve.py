"""Continuous-batching layout server.

Jobs (a graph, initial positions, a seed) arrive at any time.  Each tick of
the server:
  1. admits waiting jobs, first come first served, while a slot is free and
     the job's peak device memory during preparation fits both the server's
     HBM budget and the free device memory (cudaMemGetInfo, read once per
     tick); the graph is copied to the device
     and prepared (snap_layout_create), and the job's reservation is then
     cut to what its handle really holds (snap_layout_device_bytes) plus its
     positions;
  2. runs ONE multi-handle epoch launch (snap_multi_epoch) that advances every
     admitted job by one epoch, each at its own epoch index;
  3. retires jobs that ran all their epochs: their positions are copied back
     to pinned host memory asynchronously, and their device memory is
     returned to the budget once the copy has completed.
A job that arrives while others are on the GPU therefore starts at the next
tick, and small jobs are not stuck behind large ones.  Per-job latency is
measured from submission to the moment its result is on the host.  A job can
be cancelled while it waits or runs (cancel): it leaves the next tick's
launch, its positions are not copied back, and its memory returns to the
budget once the work already queued for it has completed.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import (MODE_HOGWILD_RED, MultiEpoch, SnapSchedule, linear_schedule, make_options, snap_layout_create,
               snap_layout_destroy, snap_layout_device_bytes, snap_memory_cached)


def estimated_bytes(n: int, nnz: int) -> int:
    """Peak device bytes of one job while it is prepared (an upper bound):
    CSR copy, orientation scan buffers and the oriented entries in both
    orders, plus positions.  Once prepared, a job holds less: its handle's
    snap_layout_device_bytes plus its positions."""
    return 48 * nnz + 40 * (n + 1) + (1 << 20)


# device memory left free for everything else on the GPU when admitting
FREE_MARGIN = 256 << 20


@dataclass
class Job:
    job_id: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    positions: np.ndarray           # (n, 2) float32 initial positions; receives the result
    seed: int
    submitted: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    epoch: int = 0
    handle: object = None
    pos_dev: object = None
    pos_host: object = None
    done_event: object = None
    reserved: int = 0
    cancelled: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


class LayoutServer:
    def __init__(self, hbm_budget: int, max_jobs: int = 256, epochs: int = 30, neg_samples: int = 3,
                 eta0: float = 1.0, mode: int = MODE_HOGWILD_RED, segment_edges: int = 0, stream=None,
                 clock=time.perf_counter):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget)
        self.max_jobs = max_jobs
        self.epochs = epochs
        self.k = neg_samples
        self.schedule: SnapSchedule = linear_schedule(eta0, epochs)
        self.opts = make_options(mode=mode, segment_edges=segment_edges)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.prep = torch.cuda.Stream()      # admission work never waits for queued ticks
        self.clock = clock
        self.multi = MultiEpoch(max_jobs)
        self.waiting: collections.deque[Job] = collections.deque()
        self.active: list[Job] = []
        self.retiring: list[Job] = []
        self.done: list[Job] = []
        self.cancelled: list[Job] = []
        self.used = 0
        self.ticks = 0
        self.updates = 0

    # -- requests -----------------------------------------------------------
    def submit(self, job: Job) -> None:
        job.submitted = self.clock()
        need = estimated_bytes(job.n, job.nnz)
        if need > self.budget:
            raise ValueError(f"job {job.job_id} needs {need} bytes, more than the whole budget")
        self.waiting.append(job)

    def cancel(self, job_id: int) -> bool:
        """Withdraws a waiting or running job; False if it is unknown or its
        result is already being copied back."""
        for job in self.waiting:
            if job.job_id == job_id:
                self.waiting.remove(job)
                job.cancelled = True
                job.finished = self.clock()
                self.cancelled.append(job)
                return True
        for job in self.active:
            if job.job_id == job_id:
                self.active.remove(job)
                job.cancelled = True
                job.done_event = self.torch.cuda.Event()
                job.done_event.record(self.stream)     # after the last tick that used the job
                self.retiring.append(job)
                return True
        return False

    def idle(self) -> bool:
        return not (self.waiting or self.active or self.retiring)

    # -- one tick -----------------------------------------------------------
    def _admit(self) -> None:
        torch = self.torch
        if not self.waiting or len(self.active) >= self.max_jobs:
            return
        # free device memory, plus what the library's pool holds for reuse
        free = torch.cuda.mem_get_info()[0] + snap_memory_cached(torch.cuda.current_device()) - FREE_MARGIN
        while self.waiting and len(self.active) < self.max_jobs:
            job = self.waiting[0]
            need = estimated_bytes(job.n, job.nnz)
            if self.used + need > self.budget or need > free:
                break
            self.waiting.popleft()
            with torch.cuda.stream(self.prep):
                job.handle = snap_layout_create(job.row_ptr, job.col_idx, None, job.n, self.opts, self.prep)
                job.pos_dev = torch.from_numpy(job.positions).pin_memory().to("cuda", non_blocking=True)
            job.pos_dev.record_stream(self.stream)
            self.stream.wait_stream(self.prep)
            job.reserved = snap_layout_device_bytes(job.handle) + job.positions.nbytes
            self.used += job.reserved
            free -= job.reserved
            job.admitted = self.clock()
            job.epoch = 0
            self.active.append(job)

    def _retire(self) -> None:
        torch = self.torch
        still = []
        for job in self.active:
            if job.epoch < self.epochs:
                still.append(job)
                continue
            job.pos_host = torch.empty(job.pos_dev.shape, dtype=torch.float32, pin_memory=True)
            job.pos_host.copy_(job.pos_dev, non_blocking=True)
            job.done_event = torch.cuda.Event()
            job.done_event.record(self.stream)
            self.retiring.append(job)
        self.active = still
        left = []
        for job in self.retiring:
            if job.done_event.query():
                if not job.cancelled:
                    job.positions[:] = job.pos_host.numpy()
                job.finished = self.clock()
                snap_layout_destroy(job.handle)
                job.handle = None
                job.pos_dev = None
                job.pos_host = None
                self.used -= job.reserved
                (self.cancelled if job.cancelled else self.done).append(job)
            else:
                left.append(job)
        self.retiring = left

    def tick(self) -> None:
        self._admit()
        if self.active:
            self.multi.epoch([(j.handle, j.pos_dev, j.epoch, self.schedule, j.seed) for j in self.active], self.k,
                             self.stream)
            for j in self.active:
                j.epoch += 1
                self.updates += j.nnz * (1 + self.k)
            self.ticks += 1
        self._retire()

    def drain(self) -> None:
        while not self.idle():
            self.tick()
            if not self.active and self.retiring:
                self.stream.synchronize()
        self.multi.check(self.stream)

    def close(self) -> None:
        for job in list(self.active) + list(self.retiring):
            if job.handle is not None:
                snap_layout_destroy(job.handle)
        self.multi.close()


def run_sequential(jobs, epochs: int = 30, neg_samples: int = 3, eta0: float = 1.0, mode: int = MODE_HOGWILD_RED,
                   stream=None, clock=time.perf_counter, arrivals=None):
    """The plain form: one job at a time, first come first served, each laid
    out completely (create, 30 epoch launches, copy back) before the next."""
    import torch
    from . import snap_layout_epochs
    stream = stream if stream is not None else torch.cuda.current_stream()
    sched = linear_schedule(eta0, epochs)
    opts = make_options(mode=mode)
    t0 = clock()
    for q, job in enumerate(jobs):
        if arrivals is not None:
            while clock() - t0 < arrivals[q]:
                pass
            job.submitted = t0 + arrivals[q]
        else:
            job.submitted = clock()
        h = snap_layout_create(job.row_ptr, job.col_idx, None, job.n, opts, stream)
        pos = torch.from_numpy(job.positions).cuda()
        job.admitted = clock()
        snap_layout_epochs(h, pos, 0, epochs, neg_samples, sched, job.seed, stream)
        job.positions[:] = pos.cpu().numpy()
        job.finished = clock()
        snap_layout_destroy(h)
    return jobs
