"""Served form: a continuous-batching sort service on one GPU.

Requests (a device tensor of keys, f64 or u64) are admitted while the bytes
they will hold on the device fit a memory budget.  K worker threads each
own a pcf context, a CUDA stream and resident device buffers.  An idle
worker takes every admitted request of one key type that fits its buffer
(first come, first served) and sorts them together with one
pcf_sort_segmented launch; requests that arrive while others are on the GPU
wait only until a worker frees up (continuous batching), and the K streams
overlap on the device.  Each result is the sorted copy of the request's
keys; it does not depend on what it was batched with, because each segment
is sorted as its own array.

Latency is measured from submission to the moment the result is ready on
the device (the worker's stream has completed the batch).
"""
import collections
import threading
import time

import numpy as np

from . import pcfsort


class Request:
    __slots__ = ("rid", "keys", "kt", "n", "out", "t_submit", "t_start", "t_done", "done",
                 "error", "nbytes")

    def __init__(self, rid, keys, kt, n=None):
        self.rid = rid
        self.keys = keys
        self.kt = kt
        self.n = keys.numel() if n is None else n
        self.out = None
        self.t_submit = time.perf_counter()
        self.t_start = None
        self.t_done = None
        self.done = threading.Event()
        self.error = None
        self.nbytes = 16 * self.n  # input copy + sorted output on the device

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_submit


class Admission:
    """Host-side admission and batching (no device work).

    submit() queues a request; it is admitted (moved to `ready`) while the
    bytes of all admitted, unfinished requests stay within `mem_budget`,
    first come first served.  take_batch() hands a worker every ready request
    of the oldest request's key type that fits `batch_keys`; complete() frees
    the bytes of a finished batch and admits waiting requests."""

    def __init__(self, mem_budget, batch_keys):
        self.mem_budget = mem_budget
        self.batch_keys = batch_keys
        self.waiting = collections.deque()
        self.ready = collections.deque()
        self.reserved = 0

    def submit(self, req):
        if req.n > self.batch_keys or req.nbytes > self.mem_budget:
            raise ValueError("request larger than a batch or the memory budget")
        self.waiting.append(req)
        self._admit()

    def _admit(self):
        while self.waiting and self.reserved + self.waiting[0].nbytes <= self.mem_budget:
            r = self.waiting.popleft()
            self.reserved += r.nbytes
            self.ready.append(r)

    def take_batch(self):
        if not self.ready:
            return []
        kt = self.ready[0].kt
        batch, total, rest = [], 0, collections.deque()
        while self.ready:
            r = self.ready.popleft()
            if r.kt == kt and total + r.n <= self.batch_keys:
                batch.append(r)
                total += r.n
            else:
                rest.append(r)
        self.ready = rest
        return batch

    def complete(self, batch):
        for r in batch:
            self.reserved -= r.nbytes
        self._admit()


class SortServer:
    """Continuous-batching sort server.

    workers      number of concurrent batches (streams) on the GPU
    mem_budget   device bytes that admitted requests may hold at once
    batch_keys   capacity of each worker's resident batch buffer (keys)
    """

    def __init__(self, device=0, workers=4, mem_budget=64 << 30, batch_keys=1 << 27,
                 tuning=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.batch_keys = batch_keys
        self.lock = threading.Condition()
        self.adm = Admission(mem_budget, batch_keys)
        self.closed = False
        self.completed = []
        self._rid = 0
        self.workers = []
        for w in range(workers):
            ctx = pcfsort.Context(device, tuning=tuning)
            ctx.reserve(batch_keys)
            stream = torch.cuda.Stream(device=self.device)
            buf_in = torch.empty(batch_keys, dtype=torch.int64, device=self.device)
            buf_out = torch.empty(batch_keys, dtype=torch.int64, device=self.device)
            th = threading.Thread(target=self._worker, args=(ctx, stream, buf_in, buf_out),
                                  daemon=True)
            self.workers.append((th, ctx))
            th.start()

    # -- client side -------------------------------------------------------
    def submit(self, keys, key_type="f64"):
        """Queues a sort of `keys` (1-D CUDA tensor, float64 or int64 holding
        u64 bits).  Returns a Request; wait on req.done."""
        with self.lock:
            r = Request(self._rid, keys, key_type)
            self.adm.submit(r)
            self._rid += 1
            self.lock.notify_all()
        return r

    def close(self):
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        for th, ctx in self.workers:
            th.join()
            ctx.close()

    # -- worker side -------------------------------------------------------
    def _worker(self, ctx, stream, buf_in, buf_out):
        torch = self.torch
        while True:
            with self.lock:
                while not self.closed and not self.adm.ready:
                    self.lock.wait()
                if self.closed and not self.adm.ready:
                    return
                batch = self.adm.take_batch()
            if not batch:
                continue
            t0 = time.perf_counter()
            offs = np.zeros(len(batch) + 1, dtype=np.uint64)
            offs[1:] = np.cumsum([r.n for r in batch])
            total = int(offs[-1])
            err = None
            try:
                with torch.cuda.stream(stream):
                    for r, o in zip(batch, offs[:-1]):
                        r.t_start = t0
                        buf_in[int(o):int(o) + r.n].copy_(r.keys.view(torch.int64),
                                                          non_blocking=True)
                    ctx.sort_segmented(buf_in[:total], offs, keys_out=buf_out[:total],
                                       key_type=batch[0].kt, seed=0, stream=stream)
                    for r, o in zip(batch, offs[:-1]):
                        out = torch.empty_like(r.keys)
                        out.view(torch.int64).copy_(buf_out[int(o):int(o) + r.n],
                                                    non_blocking=True)
                        r.out = out
            except Exception as e:  # reported per request, the server keeps going
                err = e
            finally:
                # nothing of this batch may still run when its buffers are reused
                stream.synchronize()
            t1 = time.perf_counter()
            with self.lock:
                for r in batch:
                    r.t_done = t1
                    r.error = err
                    self.completed.append(r)
                self.adm.complete(batch)
                self.lock.notify_all()
            for r in batch:
                r.done.set()


def latency_summary(requests):
    lat = np.array([r.latency for r in requests if r.latency is not None])
    if lat.size == 0:
        return {}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "count": int(lat.size)}
