"""Continuous-batching server for the visibility-bitmask gather.

Requests name a G-buffer that stays resident on the device and carry their own parameters
(slices, steps, sector count ...).  The loop admits arrived requests into the next batch as
soon as an in-flight slot and output memory are free, launches each batch with
``ssilvb_gather_batch`` on one of several streams (so batches overlap on the GPU), and
takes each request's completion time on the host clock when it first sees the batch's event
complete.  Output memory comes from one device arena with a first-fit free list; a request
waits while its outputs do not fit.  Requests of one batch share what ``ssilvb_gather_batch``
requires them to share: sector count, storage format, infinite or finite thickness and step
mode.

Admission (``LatencyAdmission``): an arriving request is admitted only if its predicted
latency fits a stated budget.  The prediction is first-in first-out service at a measured
rate: the time it has already waited, plus the predicted time of all admitted, unfinished
work, plus its own work (samples = 2 N_d N_s per pixel), divided by the rate, which starts
from a calibration and follows completed work.  A request predicted to miss the budget is
shed at arrival and counted.  Without a budget, a flat bound on the requests in the system
(queued or on the GPU) sheds arrivals beyond it.

Completed requests are handed to ``on_done(req, out0, out1)`` with views of their outputs.
Work the callback enqueues on the current CUDA stream (a copy, say) is ordered before any later
launch that reuses that memory; work it enqueues elsewhere must finish before it returns.

``PlainServer`` is the naive baseline: one request at a time, one ``ssilvb_gather`` launch
and one host synchronisation per request, under the same admission rule and the same
host-side completion clock.
"""
from __future__ import annotations

import bisect
import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    key: object             # resident G-buffer key
    params: object          # scenegen.Params-like (num_slices, steps_per_side, sector_count, ...)
    noise: np.ndarray | None = None
    sh: np.ndarray | None = None


@dataclass
class Stats:
    served: int = 0
    dropped: int = 0        # shed at arrival (predicted to miss the budget, or beyond the bound)
    within_budget: int = 0  # served with latency <= budget (all served when there is no budget)
    budget_ms: float | None = None
    samples_within_budget: int = 0
    latencies_ms: list = field(default_factory=list)
    wall_s: float = 0.0
    batches: int = 0
    max_inflight_seen: int = 0
    samples: int = 0

    def summary(self):
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"served": self.served, "shed": self.dropped, "within_budget": self.within_budget,
                "budget_ms": self.budget_ms,
                "frames_per_s": self.served / self.wall_s if self.wall_s > 0 else 0.0,
                "goodput_frames_per_s": self.within_budget / self.wall_s if self.wall_s > 0 else 0.0,
                "gsamples_per_s": self.samples / self.wall_s / 1e9 if self.wall_s > 0 else 0.0,
                "goodput_gsamples_per_s": self.samples_within_budget / self.wall_s / 1e9 if self.wall_s > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()), "mean_ms": float(lat.mean()), "batches": self.batches,
                "max_batches_in_flight": self.max_inflight_seen, "wall_s": self.wall_s}


def request_samples(H, W, prm):
    """Samples of one request: 2 N_d N_s per pixel."""
    return H * W * 2 * prm.num_slices * prm.steps_per_side


class LatencyAdmission:
    """Admission by predicted completion time under first-in first-out service.

    budget_s: the latency budget (None: no latency test); max_in_system: a bound on the admitted
    requests not yet complete (None: no bound).
    rate: predicted service rate in samples/s (a calibration); observe() moves it toward the
    rate of completed work (exponential average with weight alpha).
    A request of `samples` that arrived at `arrival` is admitted at time `now` iff
        (now - arrival) + (backlog + samples) / rate + granularity_s <= budget_s,
    backlog being the samples of every admitted request not yet complete, and granularity_s the
    longest a request can wait for work launched together with it to finish (a batch's span)."""

    def __init__(self, budget_s=None, rate=4e11, alpha=0.2, max_in_system=256, granularity_s=0.0):
        self.budget_s, self.rate, self.alpha, self.max_in_system = budget_s, float(rate), alpha, max_in_system
        self.granularity_s = granularity_s
        self.backlog = 0
        self.in_system = 0

    def predicted_latency(self, now, arrival, samples):
        return (now - arrival) + (self.backlog + samples) / self.rate + self.granularity_s

    def admit(self, now, arrival, samples):
        ok = self.max_in_system is None or self.in_system < self.max_in_system
        if ok and self.budget_s is not None:
            ok = self.predicted_latency(now, arrival, samples) <= self.budget_s
        if ok:
            self.backlog += samples
            self.in_system += 1
        return ok

    def done(self, samples):
        self.backlog -= samples
        self.in_system -= 1

    def observe(self, samples, service_s):
        """Completed work: `samples` took `service_s` of service (time since the later of its start and
        the previous completion)."""
        if service_s > 0 and samples > 0:
            self.rate = (1.0 - self.alpha) * self.rate + self.alpha * (samples / service_s)


class ResidentPool:
    """G-buffers resident on the device, by key: (depth, normal, radiance, camera)."""

    def __init__(self, device="cuda"):
        self.device = device
        self.items = {}

    def add(self, key, gbuf, interleaved=False):
        """Make gbuf resident.  interleaved: store FP16 normal and radiance as one interleaved plane
        (F16X8; the radiance entry is then None)."""
        import torch
        d = torch.from_numpy(np.ascontiguousarray(gbuf.depth)).to(self.device)
        if interleaved:
            n = torch.from_numpy(gbuf.interleaved_f16()).to(self.device)
            r = None
        else:
            n = torch.from_numpy(np.ascontiguousarray(gbuf.normal)).to(self.device)
            r = torch.from_numpy(np.ascontiguousarray(gbuf.radiance)).to(self.device)
        self.items[key] = (d, n, r, gbuf.camera)

    def shape(self, key):
        return tuple(self.items[key][0].shape)


class OutputArena:
    """First-fit allocator over one device buffer (256-byte aligned blocks)."""

    ALIGN = 256

    def __init__(self, nbytes, device="cuda"):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.size = nbytes
        self.free = [(0, nbytes)]  # sorted (offset, size)

    def alloc(self, nbytes):
        nbytes = (nbytes + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for i, (off, sz) in enumerate(self.free):
            if sz >= nbytes:
                if sz == nbytes:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + nbytes, sz - nbytes)
                return off, nbytes
        return None

    def release(self, off, nbytes):
        i = bisect.bisect(self.free, (off, 0))
        self.free.insert(i, (off, nbytes))
        # merge neighbours
        merged = []
        for o, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((o, s))
        self.free = merged

    def view(self, off, H, W):
        import torch
        return self.buf[off:off + H * W * 16].view(torch.float32).view(H, W, 4)

    def view_masks(self, off, prm, H, W):
        """Slice bitmasks [N_d, H, W, words] int32 at byte offset off (words = N_b / 32)."""
        import torch
        words = prm.sector_count // 32
        n = prm.num_slices * H * W * words * 4
        return self.buf[off:off + n].view(torch.int32).view(prm.num_slices, H, W, words)


def _mask_bytes(H, W, prm):
    return prm.num_slices * H * W * (prm.sector_count // 32) * 4


def _out_bytes(H, W, prm, with_masks=False):
    return H * W * 16 * (2 if prm.ambient_cones > 0 else 1) + (_mask_bytes(H, W, prm) if with_masks else 0)


def _batch_key(pool, req):
    """What the frames of one ssilvb_gather_batch call must share: sector count, storage format (dtype
    and components of the normal plane: 8 for the interleaved FP16 layout), infinite thickness, step
    mode."""
    n = pool.items[req.key][1]
    return (req.params.sector_count, str(n.dtype), int(n.shape[-1]), math.isinf(req.params.thickness),
            int(getattr(req.params, "step_mode", 0)))


class Server:
    """Continuous batching: batches of arrived requests, several in flight on separate streams."""

    def __init__(self, ctx, pool, arena_bytes=1 << 31, max_inflight=4, max_batch=16, max_queue=256, streams=3,
                 budget_ms=None, rate=4e11, batch_ms=None, with_masks=False):
        """batch_ms: cap on a batch's predicted GPU time (at least one request per batch); None = no cap.
        With a budget, a request may also wait for the rest of its batch, so admission adds batch_ms.
        with_masks: each request also gets its slice bitmasks, and on_done(req, out0, out1, masks)."""
        import torch
        self.ctx, self.pool = ctx, pool
        self.arena = OutputArena(arena_bytes, pool.device)
        self.max_inflight, self.max_batch, self.max_queue = max_inflight, max_batch, max_queue
        self.budget_ms, self.rate, self.batch_ms = budget_ms, rate, batch_ms
        self.with_masks = with_masks
        self.streams = [torch.cuda.Stream() for _ in range(streams)]

    def run(self, requests, on_done=None, timeout_s=120.0):
        import torch
        st = Stats(budget_ms=self.budget_ms)
        span_s = 0.0 if self.batch_ms is None else self.batch_ms / 1e3
        adm = LatencyAdmission(None if self.budget_ms is None else self.budget_ms / 1e3, self.rate,
                               max_in_system=self.max_queue, granularity_s=span_s)
        budget_s = math.inf if self.budget_ms is None else self.budget_ms / 1e3
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = collections.deque()
        inflight = collections.deque()  # (event, t_launch, samples, [(req, off, nbytes, out0, out1, samples)])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        i, si = 0, 0
        last_done = 0.0
        while i < len(reqs) or pending or inflight:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise RuntimeError("serving run exceeded its time limit")
            while i < len(reqs) and reqs[i].arrival <= now:
                req = reqs[i]
                H, W = self.pool.shape(req.key)
                # a request whose outputs exceed the whole arena could never be launched: shed it
                fits = _out_bytes(H, W, req.params, self.with_masks) <= self.arena.size
                if fits and adm.admit(now, req.arrival, request_samples(H, W, req.params)):
                    pending.append(req)
                else:
                    st.dropped += 1
                i += 1
            # completions, in launch order, timed when the host first sees them
            while inflight and inflight[0][0].query():
                ev, t_launch, bsamples, items = inflight.popleft()
                t_done = time.perf_counter() - t0
                adm.observe(bsamples, t_done - max(t_launch, last_done))
                last_done = t_done
                for req, off, nb_, o0, o1, mk, smp in items:
                    lat = t_done - req.arrival
                    st.latencies_ms.append(lat * 1e3)
                    st.served += 1
                    st.within_budget += int(lat <= budget_s)
                    st.samples_within_budget += smp if lat <= budget_s else 0
                    adm.done(smp)
                    if on_done is not None:
                        if self.with_masks:
                            on_done(req, o0, o1, mk)
                        else:
                            on_done(req, o0, o1)
                    self.arena.release(off, nb_)
            # admit and launch the next batch
            if pending and len(inflight) < self.max_inflight:
                head_key = _batch_key(self.pool, pending[0])
                batch, keep, frames = [], None, []
                skipped = collections.deque()
                cap = math.inf if self.batch_ms is None else adm.rate * self.batch_ms / 1e3
                work = 0
                while pending and len(batch) < self.max_batch:
                    req = pending.popleft()
                    if _batch_key(self.pool, req) != head_key:
                        skipped.append(req)
                        continue
                    H, W = self.pool.shape(req.key)
                    if batch and work + request_samples(H, W, req.params) > cap:
                        skipped.append(req)  # the batch's span is full: the request leads the next one
                        break
                    work += request_samples(H, W, req.params)
                    nbytes = _out_bytes(H, W, req.params, self.with_masks)
                    got = self.arena.alloc(nbytes)
                    if got is None:  # wait for memory: keep the request at its place in the queue
                        skipped.append(req)
                        break
                    off, nb_ = got
                    o0 = self.arena.view(off, H, W)
                    o1 = self.arena.view(off + H * W * 16, H, W) if req.params.ambient_cones > 0 else None
                    mk = None
                    if self.with_masks:
                        mk = self.arena.view_masks(off + _out_bytes(H, W, req.params), req.params, H, W)
                    d, n, r, cam = self.pool.items[req.key]
                    f, keep = self.ctx.frame(d, n, r, cam, req.params, o0, o1, mk, noise=req.noise, sh=req.sh,
                                             keep=keep)
                    frames.append(f)
                    batch.append((req, off, nb_, o0, o1, mk, request_samples(H, W, req.params)))
                while skipped:
                    pending.appendleft(skipped.pop())
                if batch:
                    s = self.streams[si % len(self.streams)]
                    si += 1
                    # work that on_done callbacks enqueued on the current stream (reading outputs whose
                    # arena blocks this batch may now reuse) runs before the batch
                    s.wait_stream(torch.cuda.current_stream())
                    try:
                        self.ctx.gather_batch(frames, stream=s)
                    except Exception:
                        for _, off, nb_, *_ in batch:  # nothing was enqueued: give the outputs back
                            self.arena.release(off, nb_)
                        raise
                    ev = torch.cuda.Event()
                    ev.record(s)
                    bsamples = sum(b[6] for b in batch)
                    inflight.append((ev, time.perf_counter() - t0, bsamples, batch))
                    st.samples += bsamples
                    st.batches += 1
                    st.max_inflight_seen = max(st.max_inflight_seen, len(inflight))
                    continue
            time.sleep(0.0001)
        st.wall_s = max(last_done, 1e-9) - (reqs[0].arrival if reqs else 0.0)
        return st


class PlainServer:
    """Naive baseline: one launch and one host synchronisation per request, in arrival order, under
    the same admission rule as Server."""

    def __init__(self, ctx, pool, max_queue=256, budget_ms=None, rate=4e11):
        self.ctx, self.pool, self.max_queue = ctx, pool, max_queue
        self.budget_ms, self.rate = budget_ms, rate
        self.outs = {}

    def _outputs(self, key, prm):
        import torch
        k = (key, prm.ambient_cones > 0)
        if k not in self.outs:
            H, W = self.pool.shape(key)
            o0 = torch.empty((H, W, 4), dtype=torch.float32, device=self.pool.device)
            o1 = torch.empty((H, W, 4), dtype=torch.float32, device=self.pool.device) if prm.ambient_cones else None
            self.outs[k] = (o0, o1)
        return self.outs[k]

    def run(self, requests, on_done=None, timeout_s=120.0):
        import torch
        st = Stats(budget_ms=self.budget_ms)
        adm = LatencyAdmission(None if self.budget_ms is None else self.budget_ms / 1e3, self.rate,
                               max_in_system=self.max_queue)
        budget_s = math.inf if self.budget_ms is None else self.budget_ms / 1e3
        reqs = sorted(requests, key=lambda r: r.arrival)
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        last_done = 0.0
        waiting = collections.deque()
        i = 0
        while i < len(reqs) or waiting:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise RuntimeError("serving run exceeded its time limit")
            while i < len(reqs) and reqs[i].arrival <= now:
                req = reqs[i]
                H, W = self.pool.shape(req.key)
                if adm.admit(now, req.arrival, request_samples(H, W, req.params)):
                    waiting.append(req)
                else:
                    st.dropped += 1
                i += 1
            if not waiting:
                time.sleep(0.0001)
                continue
            req = waiting.popleft()
            d, n, r, cam = self.pool.items[req.key]
            o0, o1 = self._outputs(req.key, req.params)
            t_start = time.perf_counter() - t0
            # the previous on_done's work on the current stream may still read these outputs
            stream.wait_stream(torch.cuda.current_stream())
            self.ctx.gather(d, n, r, cam, req.params, o0, o1, None, noise=req.noise, sh=req.sh, stream=stream)
            stream.synchronize()
            t_done = time.perf_counter() - t0
            H, W = self.pool.shape(req.key)
            smp = request_samples(H, W, req.params)
            adm.observe(smp, t_done - max(t_start, last_done))
            adm.done(smp)
            last_done = t_done
            lat = t_done - req.arrival
            st.latencies_ms.append(lat * 1e3)
            st.served += 1
            st.within_budget += int(lat <= budget_s)
            st.samples_within_budget += smp if lat <= budget_s else 0
            st.samples += smp
            if on_done is not None:
                on_done(req, o0, o1)
        st.wall_s = max(last_done, 1e-9) - (reqs[0].arrival if reqs else 0.0)
        st.batches = st.served
        return st


def poisson_requests(seed, n, mean_gap_s, keys, sizes_of, nd_range=(1, 8), nb_choices=(32, 64),
                     ns_choices=(8, 16, 32), radius=2.0, thickness=0.5):
    """A seeded Poisson arrival stream over resident G-buffer keys with per-request parameters."""
    import scenegen
    u = scenegen.uniform(seed, 6 * n)
    t = 0.0
    out = []
    noise = scenegen.ign_table()
    for k in range(n):
        t += float(-mean_gap_s * np.log(max(1.0 - u[6 * k], 1e-12)))
        key = keys[min(int(u[6 * k + 1] * len(keys)), len(keys) - 1)]
        nd = nd_range[0] + min(int(u[6 * k + 2] * (nd_range[1] - nd_range[0] + 1)), nd_range[1] - nd_range[0])
        nb = nb_choices[min(int(u[6 * k + 3] * len(nb_choices)), len(nb_choices) - 1)]
        ns = ns_choices[min(int(u[6 * k + 4] * len(ns_choices)), len(ns_choices) - 1)]
        prm = scenegen.Params(num_slices=nd, steps_per_side=ns, radius=radius, thickness=thickness, sector_count=nb)
        out.append(Request(k, t, key, prm, noise, None))
    return out
