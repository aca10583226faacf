"""Served form: a continuous-batching sort service on one GPU.

Requests (a device tensor of keys, f64 or u64) are admitted while their
results fit in a resident result pool on the device.  The pool is allocated
once, when the server starts, at the smaller of the memory budget and the
device memory then free (cudaMemGetInfo, less a headroom), so admission
follows the memory the device really has.  Each admitted request owns a
slice of the pool until the client releases it.  K worker threads each own a
pcf context, a CUDA stream and resident batch buffers.  An idle worker takes
every admitted request of one key type that fits its buffers (first come,
first served) and sorts them together with one pcf_sort_segmented launch;
requests that arrive while others are on the GPU wait only until a worker
frees up (continuous batching), and the K streams overlap on the device.
Each result is the sorted copy of the request's keys; it does not depend on
what it was batched with, because each segment is sorted as its own array.

Stream order: submit() records an event on the caller's current stream, and
the worker's stream waits on it before reading the keys, so keys produced
by kernels still in flight are read only once they are complete.  A result
is complete on the device when its request's `done` is set (the worker's
stream has finished the batch).

Latency is measured from submission to the moment the result is ready on
the device.
"""
import bisect
import collections
import threading
import time

import numpy as np

from . import pcfsort

KEY_BYTES = 8


class Request:
    __slots__ = ("rid", "keys", "kt", "n", "out", "t_submit", "t_start", "t_done", "done",
                 "error", "nbytes", "slot", "ready_event", "server")

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
        self.nbytes = KEY_BYTES * self.n  # its result, held in the pool until released
        self.slot = None                  # offset of the result in the pool (keys)
        self.ready_event = None
        self.server = None

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_submit

    def release(self):
        """Gives the result's pool slice back (the result tensor becomes
        invalid).  Safe to call more than once."""
        if self.server is not None:
            self.server.release(self)


class ResultPool:
    """First-fit allocation of key slices from a fixed range [0, capacity)
    (host-side bookkeeping of the resident device arena)."""

    def __init__(self, capacity):
        self.capacity = capacity
        self.starts = [0]        # free blocks, sorted by start
        self.sizes = [capacity]

    def alloc(self, n):
        for i, sz in enumerate(self.sizes):
            if sz >= n:
                off = self.starts[i]
                if sz == n:
                    del self.starts[i]
                    del self.sizes[i]
                else:
                    self.starts[i] += n
                    self.sizes[i] -= n
                return off
        return None

    def release(self, off, n):
        i = bisect.bisect_left(self.starts, off)
        self.starts.insert(i, off)
        self.sizes.insert(i, n)
        # merge with the next block, then with the previous one
        if i + 1 < len(self.starts) and self.starts[i] + self.sizes[i] == self.starts[i + 1]:
            self.sizes[i] += self.sizes.pop(i + 1)
            self.starts.pop(i + 1)
        if i > 0 and self.starts[i - 1] + self.sizes[i - 1] == self.starts[i]:
            self.sizes[i - 1] += self.sizes.pop(i)
            self.starts.pop(i)

    def free_keys(self):
        return sum(self.sizes)


class Admission:
    """Host-side admission and batching (no device work).

    submit() queues a request; it is admitted (moved to `ready`) while the
    bytes of all admitted, unreleased requests stay within `mem_budget` and
    its result finds room in the pool, first come first served (a request
    that does not fit holds back those behind it).  take_batch() hands a
    worker every ready request of the oldest request's key type that fits
    `batch_keys`.  Without a pool the results belong to the clients and a
    request's bytes are freed when its batch completes; with one they are
    freed by release()."""

    def __init__(self, mem_budget, batch_keys, pool=None):
        self.mem_budget = mem_budget
        self.batch_keys = batch_keys
        self.pool = pool
        self.waiting = collections.deque()
        self.ready = collections.deque()
        self.reserved = 0

    def submit(self, req):
        cap = self.mem_budget if self.pool is None else min(self.mem_budget,
                                                            KEY_BYTES * self.pool.capacity)
        if req.n > self.batch_keys or req.nbytes > cap:
            raise ValueError("request larger than a batch or the memory budget")
        self.waiting.append(req)
        self._admit()

    def _admit(self):
        while self.waiting:
            r = self.waiting[0]
            if self.reserved + r.nbytes > self.mem_budget:
                break
            if self.pool is not None:
                slot = self.pool.alloc(r.n)
                if slot is None:
                    break
                r.slot = slot
            self.waiting.popleft()
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
        if self.pool is None:
            for r in batch:
                self.reserved -= r.nbytes
            self._admit()

    def release(self, req):
        if self.pool is None or req.slot is None:
            return
        self.pool.release(req.slot, req.n)
        req.slot = None
        self.reserved -= req.nbytes
        self._admit()


class SortServer:
    """Continuous-batching sort server.

    workers      number of concurrent batches (streams) on the GPU
    mem_budget   device bytes that unreleased results may hold at once (the
                 result pool is the smaller of this and the free device
                 memory at start, less `headroom` bytes)
    batch_keys   capacity of each worker's resident batch buffers (keys)
    """

    def __init__(self, device=0, workers=4, mem_budget=64 << 30, batch_keys=1 << 27,
                 tuning=None, headroom=4 << 30):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.batch_keys = batch_keys
        self.lock = threading.Condition()
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
            self.workers.append((ctx, stream, buf_in, buf_out))
        # the resident result pool, sized by the memory the device has free now
        free, _ = torch.cuda.mem_get_info(self.device)
        pool_bytes = max(0, min(mem_budget, free - headroom))
        self.pool_keys = pool_bytes // KEY_BYTES
        if self.pool_keys < 1:
            raise RuntimeError("no device memory left for the result pool")
        self.pool_buf = torch.empty(self.pool_keys, dtype=torch.int64, device=self.device)
        self.adm = Admission(mem_budget, batch_keys, pool=ResultPool(self.pool_keys))
        self.threads = []
        for w in self.workers:
            th = threading.Thread(target=self._worker, args=w, daemon=True)
            self.threads.append(th)
            th.start()

    # -- client side -------------------------------------------------------
    def submit(self, keys, key_type="f64"):
        """Queues a sort of `keys` (1-D CUDA tensor, float64 or int64 holding
        u64 bits), ordered after the work already queued on the caller's
        current stream.  Returns a Request: wait on req.done, read req.out,
        then req.release()."""
        torch = self.torch
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream(keys.device))
        with self.lock:
            r = Request(self._rid, keys, key_type)
            r.ready_event = ev
            r.server = self
            self.adm.submit(r)
            self._rid += 1
            self.lock.notify_all()
        return r

    def release(self, req):
        with self.lock:
            req.out = None
            self.adm.release(req)
            self.lock.notify_all()

    def close(self):
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        for th in self.threads:
            th.join()
        for ctx, _, _, _ in self.workers:
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
                        stream.wait_event(r.ready_event)
                        buf_in[int(o):int(o) + r.n].copy_(r.keys.view(torch.int64),
                                                          non_blocking=True)
                    ctx.sort_segmented(buf_in[:total], offs, keys_out=buf_out[:total],
                                       key_type=batch[0].kt, seed=0, stream=stream)
                    for r, o in zip(batch, offs[:-1]):
                        dst = self.pool_buf[r.slot:r.slot + r.n]
                        dst.copy_(buf_out[int(o):int(o) + r.n], non_blocking=True)
                        r.out = dst if r.kt != "f64" else dst.view(torch.float64)
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
                    r.keys = None  # the input is no longer needed
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
