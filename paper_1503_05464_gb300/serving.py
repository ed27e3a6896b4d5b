"""Serving loop: compress + solve requests with continuous batching.

Each request brings a dense matrix (here a Schur complement of a 3D Laplacian,
n = k^2) and a schedule of right-hand-side batches.  The loop

* admits an arrived request as soon as its estimated device memory fits the
  HBM budget, and submits its compression to a running incremental batch
  (hss_batch_submit): requests that arrive while others are being compressed
  join the same per-level launches at the next round;
* advances the batch one round at a time (one tree level of every job);
* hands each finished compression to a second host thread with its own CUDA
  stream, which factors the newly finished forms together
  (hss_factor_batched), keeps them resident, serves every due right-hand-side
  batch together (hss_solve_batched) and releases a request's form after its
  last solve -- so factorizations and solves overlap the compression rounds
  on the device instead of stalling them;
* frees each input matrix as soon as its compression is done.

It reports p50/p99 latencies (arrival to first solution, and per solve batch)
and throughput.  All GPU work runs in libhss; this module only schedules.
"""
from __future__ import annotations

import heapq
import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import hss as H


@dataclass
class Request:
    rid: int
    k: int                          # grid size: n = k^2
    arrival: float                  # seconds after start
    solves: list                    # [(seconds after compression done, nrhs)]
    scale: float = 1.0
    # filled by the server
    A: torch.Tensor | None = None
    ticket: int = -1
    handle: H.HSS | None = None
    t_admit: float = math.nan
    t_compressed: float = math.nan
    t_first_solution: float = math.nan
    reserved: int = 0
    resident: int = 0
    solves_left: int = 0
    ranks: int = 0

    @property
    def n(self):
        return self.k * self.k


def poisson_requests(count, rate, ks, seed, max_solves=3, nrhs_range=(1, 64)):
    """`count` requests, exponential inter-arrival times at `rate` per second,
    grid sizes drawn from `ks`, 1..max_solves solve batches of 1..64 RHS."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        ns = int(rng.integers(1, max_solves + 1))
        solves = sorted((float(rng.exponential(0.05)), int(rng.integers(nrhs_range[0], nrhs_range[1] + 1)))
                        for _ in range(ns))
        out.append(Request(i, int(rng.choice(ks)), t, solves, scale=float(1.0 + 0.1 * rng.random())))
    return out


def estimate_bytes(n, opts, esz=4):
    """Peak device memory of one compression: the matrix (twice when its rows
    are not 16-byte aligned: the tensor-core sampling reads a padded copy),
    the samples, the column-sample partial slab of one pass, and the
    resident form."""
    d = max(opts.d0, 64) * 4
    a = n * n * esz
    if esz == 4 and n % 4 != 0 and opts.sample_mode != 0:
        a += n * ((n + 3) // 4 * 4) * esz
    samples = 3 * n * d * esz
    slab = ((n + 127) // 128) * ((opts.d0 + 63) // 64) * n * 64 * esz
    return a + samples + slab


@dataclass
class ServeStats:
    requests: int = 0
    solves: int = 0
    rhs: int = 0
    wall_s: float = 0.0
    request_latency: list = field(default_factory=list)
    solve_latency: list = field(default_factory=list)
    compress_latency: list = field(default_factory=list)
    peak_reserved: int = 0
    max_inflight: int = 0

    def summary(self):
        def pct(v, q):
            return float(np.percentile(v, q)) if v else None
        return {
            "requests": self.requests, "solves": self.solves, "rhs": self.rhs,
            "wall_s": self.wall_s,
            "request_p50_s": pct(self.request_latency, 50),
            "request_p99_s": pct(self.request_latency, 99),
            "solve_p50_s": pct(self.solve_latency, 50),
            "solve_p99_s": pct(self.solve_latency, 99),
            "compress_p50_s": pct(self.compress_latency, 50),
            "solves_per_s": self.solves / self.wall_s if self.wall_s else None,
            "rhs_per_s": self.rhs / self.wall_s if self.wall_s else None,
            "peak_reserved_gb": self.peak_reserved / 1e9,
            "max_inflight": self.max_inflight,
        }


class Server:
    def __init__(self, make_matrix, opts, budget_bytes, stream=None, keep_handles=False,
                 lane_split_n=None):
        self.make_matrix = make_matrix          # k -> device template matrix
        self.lane_split_n = lane_split_n        # order from which requests get their own lane
        self.opts = opts
        self.budget = budget_bytes
        self.stream = stream
        self.keep = keep_handles
        self.templates = {}
        self.done = []

    def _template(self, k):
        if k not in self.templates:
            self.templates[k] = self.make_matrix(k)
        return self.templates[k]

    def run(self, requests):
        st = ServeStats(requests=len(requests))
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:                     # generate inputs before the clock starts
            self._template(r.k)
        torch.cuda.synchronize()
        lock = threading.Lock()
        acct = {"used": 0, "inflight": 0}
        finished = queue.Queue()              # compressed requests for the factor thread
        errors = []
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        # lanes: requests of order >= lane_split_n compress in a batch of their
        # own, stepped by its own thread on its own stream, so that the small
        # requests' rounds do not wait for a large request's level work
        nlanes = 2 if self.lane_split_n else 1
        lane_q = [queue.Queue() for _ in range(nlanes)]
        admitting = threading.Event()
        admitting.set()
        due = []                              # heap of (time, seq, request, nrhs)
        factor_done = threading.Event()
        lanes_done = [threading.Event() for _ in range(nlanes)]
        lanes = [threading.Thread(target=self._lane_thread,
                                  args=(q, lane_q[q], finished, st, lock, acct, now, errors,
                                        admitting, lanes_done[q]), daemon=True)
                 for q in range(nlanes)]
        workers = [threading.Thread(target=self._factor_thread,
                                    args=(finished, due, lock, acct, now, errors, factor_done),
                                    daemon=True),
                   threading.Thread(target=self._solve_thread,
                                    args=(due, st, lock, acct, now, errors, factor_done),
                                    daemon=True)]
        for w in lanes + workers:
            w.start()
        try:
            while pending:
                if errors:
                    raise errors[0]
                t = now()
                # admission: arrived requests whose estimate fits the budget
                while pending and pending[0].arrival <= t:
                    r = pending[0]
                    need = estimate_bytes(r.n, self.opts)
                    with lock:
                        if acct["used"] + need > self.budget and (acct["inflight"] or acct["used"] > 0):
                            break
                        acct["used"] += need
                        acct["inflight"] += 1
                        st.peak_reserved = max(st.peak_reserved, acct["used"])
                        st.max_inflight = max(st.max_inflight, acct["inflight"])
                    pending.pop(0)
                    r.A = self._template(r.k) * r.scale
                    torch.cuda.current_stream().synchronize()   # r.A ready for any lane's stream
                    r.reserved = need
                    r.t_admit = now()
                    lane = 1 if self.lane_split_n and r.n >= self.lane_split_n else 0
                    lane_q[lane].put(r)
                wait = (pending[0].arrival - now()) if pending else 0.0
                time.sleep(max(0.0, min(wait, 0.002)))
        finally:
            admitting.clear()                 # no more requests for the lanes
            for q in lane_q:
                q.put(None)
            for w in lanes:
                w.join()
            finished.put(None)                # no more compressions
            for w in workers:
                w.join()
        if errors:
            raise errors[0]
        st.wall_s = now()
        return st

    def _lane_thread(self, lane, inbox, finished, st, lock, acct, now, errors, admitting, done):
        """Compresses the requests of one lane in one incremental batch on
        its own stream: submits what the admission sent, runs one round of
        every compression in flight, hands finished ones on."""
        stream = self.stream if lane == 0 and self.stream is not None else torch.cuda.Stream()
        batch = H.HssBatch(torch.float32, stream)
        inflight = {}
        closing = False
        try:
            while True:
                while True:
                    try:
                        r = inbox.get(timeout=0.002) if not inflight and not closing else \
                            inbox.get_nowait()
                    except queue.Empty:
                        break
                    if r is None:
                        closing = True
                        break
                    r.ticket = batch.submit(r.A, self.opts)
                    inflight[r.ticket] = r
                if not inflight:
                    if closing:
                        return
                    continue
                batch.step()
                for ticket in list(inflight):
                    h, status = batch.take(ticket)
                    if status == H.HSS_ERR_STATE:
                        continue
                    r = inflight.pop(ticket)
                    if h is None:
                        raise H.HssError(status, f"request {r.rid} failed")
                    r.handle = h
                    r.t_compressed = now()
                    st.compress_latency.append(r.t_compressed - r.arrival)
                    r.A = None                # the input is no longer needed
                    with lock:
                        acct["inflight"] -= 1
                    finished.put(r)
        except Exception as e:                # reported by the admitting thread
            errors.append(e)
        finally:
            batch.close()
            done.set()

    def _factor_thread(self, finished, due, lock, acct, now, errors, factor_done):
        """Factors the finished compressions on its own stream, all those
        waiting at once (one launch per level round), and schedules their
        right-hand sides."""
        stream = torch.cuda.Stream()
        seq = 0
        closing = False
        try:
            while not closing:
                fresh = []
                r = finished.get()                # wait for the next compression
                while True:
                    if r is None:
                        closing = True
                    else:
                        fresh.append(r)
                    try:
                        r = finished.get_nowait()
                    except queue.Empty:
                        break
                if not fresh:
                    continue
                sts = H.hss_factor_batched([q.handle for q in fresh], stream=stream)
                for q, status in zip(fresh, sts):
                    if status != H.HSS_OK:
                        raise H.HssError(status, f"request {q.rid}: factorization failed")
                    info = H.hss_info(q.handle)
                    q.ranks = max(info["max_rank_r"], info["max_rank_c"])
                    q.resident = info["bytes_hss"] + info["bytes_ulv"]
                    q.solves_left = len(q.solves)
                    t = now()
                    with lock:
                        acct["used"] += q.resident - q.reserved
                        for off, nrhs in q.solves:
                            heapq.heappush(due, (t + off, seq, q, nrhs))
                            seq += 1
        except Exception as e:                # reported by the admitting thread
            errors.append(e)
        finally:
            factor_done.set()

    def _solve_thread(self, due, st, lock, acct, now, errors, factor_done):
        """Serves every due right-hand side on its own stream, all those due
        at once (one launch per sweep round), and releases finished requests."""
        stream = torch.cuda.Stream()
        try:
            with torch.cuda.stream(stream):
                while True:
                    t = now()
                    batchq = []
                    with lock:
                        while due and due[0][0] <= t:
                            batchq.append(heapq.heappop(due))
                        nxt = due[0][0] if due else None
                    if batchq:
                        Bs = []
                        for _, _, r, nrhs in batchq:
                            g = torch.Generator(device="cuda").manual_seed(1000 * r.rid + nrhs)
                            Bs.append(torch.randn(r.n, nrhs, device="cuda", generator=g))
                        Xs, sts = H.hss_solve_batched([q[2].handle for q in batchq], Bs,
                                                      stream=stream)
                        stream.synchronize()
                        tf = now()
                        for (tdue, _, r, nrhs), status in zip(batchq, sts):
                            if status != H.HSS_OK:
                                raise H.HssError(status, f"request {r.rid}: solve failed")
                            st.solve_latency.append(tf - tdue)
                            st.solves += 1
                            st.rhs += nrhs
                            if math.isnan(r.t_first_solution):
                                r.t_first_solution = tf
                                st.request_latency.append(tf - r.arrival)
                            r.solves_left -= 1
                            if r.solves_left == 0:
                                with lock:
                                    acct["used"] -= r.resident
                                if self.keep:
                                    self.done.append(r)
                                else:
                                    r.handle.close()
                                    r.handle = None
                        del Xs, Bs
                        continue
                    if nxt is None and factor_done.is_set():
                        with lock:
                            if not due:
                                return
                        continue
                    wait = (nxt - now()) if nxt is not None else 0.001
                    time.sleep(max(0.0, min(wait, 0.001)))
        except Exception as e:                # reported by the admitting thread
            errors.append(e)
