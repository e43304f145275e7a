"""Continuous-batching request loop over independent channel runs.

Each request is one channel run (its own box, grid, Reynolds number, seeded
initial field and length in substeps).  Requests arrive over time; the loop
admits a waiting request as soon as a slot is free and its device footprint
(``chan_footprint_bytes``) fits the HBM budget, keeps every admitted run's
state on the device, and advances all admitted runs concurrently, each on
its own CUDA stream, one RK3 step (a graph replay of three substeps) at a
time, with at most two steps of a run in flight.  Work of different runs
overlaps on the GPU; a run's arithmetic does not depend on what else runs
(every kernel is deterministic and its launch shape depends on the run's own
sizes only), so a result is bitwise the same alone and in the mix.

With ``packed=True`` the admitted runs of one precision advance together:
one RK3 step of all of them is one launch per kernel (``chan_batch_step``,
graph-replayed), on a single batch stream; a run's last partial step runs on
its own stream.  With ``packed="persistent"`` every admitted run of a precision (up to
16 per batch) advances in persistent launches (``chan_batch_step_each``) of up to
``persist_chunk`` substeps of each run: the launch's CTAs take the blocks of any run whose
previous stage is done, so the phases of different runs overlap and each run goes on to
its next substep without a batch-wide boundary; a run's last partial step is part of a
launch too.  There a run's step latency is its launch's device time per RK3 step the
launch advanced it by.

Per-step latency is the device time between CUDA events recorded around each
RK3 step (contention included; in packed mode the packed step's time counts
once for every run in it); request latency is arrival to completion on the
host clock.

Every admitted run issues on its own stream: a process that serves many runs should set
CUDA_DEVICE_MAX_CONNECTIONS (e.g. 32) before it creates its CUDA context, since with the
default 8 hardware work queues the streams alias and their work serialises (bench.py does).

A newly admitted run is built (tables, state upload, launch-shape tuning) on
a set-up thread while the loop keeps issuing the other runs' steps; the run
holds its slot and its memory from admission on and starts stepping once its
set-up is done.  A retired run's packed batches are dropped with it.
"""
import collections
import concurrent.futures
import math
import time

import numpy as np

from . import CHAN_PREC_FP64, Channel, ChannelBatch, footprint_bytes


class Request:
    """One channel run to serve."""

    def __init__(self, rid, t_arrival, re_tau, Lx, Lz, Nx, Ny, Nz, dt, nsub, seed, precision=CHAN_PREC_FP64):
        self.rid, self.t_arrival = rid, float(t_arrival)
        self.re_tau, self.Lx, self.Lz = float(re_tau), float(Lx), float(Lz)
        self.Nx, self.Ny, self.Nz, self.dt = int(Nx), int(Ny), int(Nz), float(dt)
        self.nsub, self.seed, self.precision = int(nsub), int(seed), int(precision)

    @property
    def points(self):
        return self.Nx * self.Ny * self.Nz

    def __repr__(self):
        return "Request(%d, t=%.3f, Re=%g, %dx%dx%d, %d substeps)" % (
            self.rid, self.t_arrival, self.re_tau, self.Nx, self.Ny, self.Nz, self.nsub)


def serving_dt(re_tau, Lx, Lz, Nx, Nz):
    """Fixed dt of a served run: min(1e-3, 0.8 sqrt(3) / (k1max 1.5 U_b + k3max 0.2 U_b)).

    U_b = 2.5 ln Re_tau + 3 (the laminar-start bulk velocity of the inputs);
    sqrt(3) is the stability limit of the explicit RK3 part on imaginary
    eigenvalues, used at 80 %.
    """
    ub = 2.5 * math.log(re_tau) + 3.0
    k1 = 2 * math.pi / Lx * (Nx // 2 - 1)
    k3 = 2 * math.pi / Lz * (Nz // 2 - 1)
    return min(1e-3, 0.8 * math.sqrt(3.0) / (k1 * 1.5 * ub + k3 * 0.2 * ub))


def poisson_requests(n, rate, seed, precision=CHAN_PREC_FP64, length=(100, 2000), res=(180.0, 395.0, 550.0),
                     nxz=(32, 64, 128), nys=(49, 97, 129), Lx=math.pi, Lz=math.pi / 2):
    """The seeded serving mix: Poisson arrivals at ``rate`` per second of minimal-box runs."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        re = float(rng.choice(res))
        Nx, Nz = int(rng.choice(nxz)), int(rng.choice(nxz))
        Ny = int(rng.choice(nys))
        nsub = int(rng.integers(length[0], length[1] + 1))
        out.append(Request(i, t[i], re, Lx, Lz, Nx, Ny, Nz, serving_dt(re, Lx, Lz, Nx, Nz), nsub,
                           seed * 1000 + i, precision))
    return out


def _pct(x, q):
    return float(np.percentile(np.asarray(x, dtype=np.float64), q)) if len(x) else None


class _Slot:
    def __init__(self, req, ch, stream, fp, t_admit):
        self.req, self.ch, self.stream, self.fp, self.t_admit = req, ch, stream, fp, t_admit
        self.remaining = req.nsub
        self.inflight = collections.deque()
        self.packed_pending = 0


class Server:
    """Admission by HBM footprint and slot count; concurrent streams; step latencies.

    ``factory(req, stream)`` builds a started channel for a request (state
    set); ``make_stream()`` and ``make_event()`` wrap torch's CUDA objects;
    ``footprint(req)`` gives its device bytes.  All four are injectable so
    that the admission and retirement logic can run without a GPU.
    """

    def __init__(self, hbm_budget, max_slots=16, chunk=3, max_inflight=2, factory=None, footprint=None,
                 make_stream=None, make_event=None, clock=time.perf_counter, idle_sleep=2e-4, packed=False,
                 make_batch=None, setup_threads=1, persist_chunk=24):
        self.hbm_budget, self.max_slots, self.chunk, self.max_inflight = int(hbm_budget), max_slots, chunk, max_inflight
        if factory is None:
            raise ValueError("a channel factory is required (see channel_factory)")
        self.factory = factory
        self.footprint = footprint or (lambda r: footprint_bytes(r.Nx, r.Ny, r.Nz, r.precision))
        self.make_stream = make_stream or _torch_stream
        self.make_event = make_event or _torch_event
        self.clock, self.idle_sleep = clock, idle_sleep
        self.packed = packed
        persistent = packed == "persistent"
        self.batch_runs = 16 if persistent else None   # runs per batch (a persistent launch holds 16)
        self.make_batch = make_batch or (lambda chans, stream: ChannelBatch(chans, stream=stream.cuda_stream,
                                                                            persistent=persistent))
        self.setup_threads = int(setup_threads)   # 0: build admitted runs on the loop's own thread
        self.persist_chunk = int(persist_chunk)    # substeps of a run per persistent launch

    def _persist_counts(self, part):
        """Substeps of each run of a persistent launch: persist_chunk (whole RK3 steps), or what
        the run has left.  (Counts in proportion to the runs' sizes served less: a small run's
        substep is not proportionally shorter, its sweeps being serial over its wall-normal
        points.)"""
        return [min(sl.remaining, self.persist_chunk) for sl in part]

    def run(self, requests, keep_results=True):
        for r in requests:
            if self.footprint(r) > self.hbm_budget:
                raise ValueError("request %d needs %d bytes, more than the whole budget" % (r.rid, self.footprint(r)))
        dev = _current_device()
        pool = (concurrent.futures.ThreadPoolExecutor(max_workers=self.setup_threads, initializer=_set_device,
                                                      initargs=(dev,))
                if self.setup_threads > 0 else None)
        try:
            return self._run(requests, keep_results, pool)
        finally:
            if pool is not None:
                pool.shutdown(wait=True)

    def _run(self, requests, keep_results, pool):
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        waiting = collections.deque()
        active, starting = [], []
        used = 0
        results, done = {}, {}
        step_ms, max_conc, conc_samples = [], 0, []
        bstream, binflight, batches, nbuilt = None, collections.deque(), {}, 0
        t0 = self.clock()
        while pending or waiting or active or starting:
            now = self.clock() - t0
            while pending and pending[0].t_arrival <= now:
                waiting.append(pending.popleft())
            progressed = False
            # admission: first come, first served, while a slot and the memory allow; the run
            # is built on the set-up thread and holds its slot and memory meanwhile
            while (waiting and len(active) + len(starting) < self.max_slots
                   and used + self.footprint(waiting[0]) <= self.hbm_budget):
                r = waiting.popleft()
                stream = self.make_stream()
                fp = self.footprint(r)
                used += fp
                t_admit = self.clock() - t0
                if pool is None:
                    active.append(_Slot(r, self.factory(r, stream), stream, fp, t_admit))
                else:
                    starting.append((r, stream, fp, t_admit, pool.submit(self.factory, r, stream)))
                progressed = True
            if starting:
                still_starting = []
                for r, stream, fp, t_admit, fut in starting:
                    if fut.done():
                        active.append(_Slot(r, fut.result(), stream, fp, t_admit))
                        progressed = True
                    else:
                        still_starting.append((r, stream, fp, t_admit, fut))
                starting = still_starting
            max_conc = max(max_conc, len(active) + len(starting))
            # persistent issue: every run with work left advances by up to persist_chunk substeps
            # in one launch per batch of a precision
            if self.packed == "persistent":
                if bstream is None:
                    bstream = self.make_stream()
                groups = collections.defaultdict(list)
                for sl in active:
                    if sl.remaining > 0:
                        groups[sl.req.precision].append(sl)
                for prec, sls in groups.items():
                    for i in range(0, len(sls), self.batch_runs):
                        part = sls[i:i + self.batch_runs]
                        if len(binflight) >= self.max_inflight:
                            break
                        key = tuple(sl.req.rid for sl in part)
                        if key not in batches:
                            batches[key] = self.make_batch([sl.ch for sl in part], bstream)
                            nbuilt += 1
                        ks = self._persist_counts(part)
                        e0, e1 = self.make_event(), self.make_event()
                        e0.record(bstream)
                        batches[key].step_each(ks)
                        e1.record(bstream)
                        binflight.append((e0, e1, list(zip(part, ks))))
                        for sl, k in zip(part, ks):
                            sl.remaining -= k
                            sl.packed_pending += 1
                        progressed = True
                while binflight and binflight[0][1].query():
                    e0, e1, ran = binflight.popleft()
                    t = e0.elapsed_time(e1)
                    for sl, k in ran:
                        sl.packed_pending -= 1
                        if k >= self.chunk:
                            step_ms.append(t * self.chunk / k)
                    progressed = True
            # packed issue: one RK3 step of every full-step run of a precision in one launch per kernel
            elif self.packed:
                if bstream is None:
                    bstream = self.make_stream()
                groups = collections.defaultdict(list)
                for sl in active:
                    if sl.remaining >= self.chunk:
                        groups[sl.req.precision].append(sl)
                parts = []
                for prec, sls in groups.items():
                    n = self.batch_runs or len(sls)
                    parts += [sls[i:i + n] for i in range(0, len(sls), n)]
                for sls in parts:
                    if len(binflight) >= self.max_inflight:
                        break
                    key = tuple(sl.req.rid for sl in sls)
                    if key not in batches:
                        batches[key] = self.make_batch([sl.ch for sl in sls], bstream)
                        nbuilt += 1
                    e0, e1 = self.make_event(), self.make_event()
                    e0.record(bstream)
                    batches[key].step(self.chunk)
                    e1.record(bstream)
                    binflight.append((e0, e1, sls))
                    for sl in sls:
                        sl.remaining -= self.chunk
                        sl.packed_pending += 1
                    progressed = True
                while binflight and binflight[0][1].query():
                    e0, e1, sls = binflight.popleft()
                    t = e0.elapsed_time(e1)
                    for sl in sls:
                        sl.packed_pending -= 1
                        step_ms.append(t)
                    progressed = True
            # issue: one RK3 step per run, up to max_inflight steps queued per stream
            for sl in active:
                if self.packed == "persistent" or (self.packed and (sl.remaining >= self.chunk or sl.packed_pending)):
                    continue
                while sl.remaining > 0 and len(sl.inflight) < self.max_inflight:
                    k = min(self.chunk, sl.remaining)
                    e0, e1 = self.make_event(), self.make_event()
                    e0.record(sl.stream)
                    sl.ch.step(k)
                    e1.record(sl.stream)
                    sl.inflight.append((e0, e1, k))
                    sl.remaining -= k
                    progressed = True
            # retire finished steps and runs
            still = []
            for sl in active:
                while sl.inflight and sl.inflight[0][1].query():
                    e0, e1, k = sl.inflight.popleft()
                    if k == self.chunk:
                        step_ms.append(e0.elapsed_time(e1))
                    progressed = True
                if sl.remaining == 0 and not sl.inflight and not sl.packed_pending:
                    # the packed batches this run was part of are of no further use; a persistent
                    # one first reports whether any of its launches ran out of polls (the run's
                    # state would then be void: ChanError)
                    for key in [k for k in batches if sl.req.rid in k]:
                        b = batches.pop(key)
                        if self.packed == "persistent" and hasattr(b, "status"):
                            b.status()
                        b.close()
                    if keep_results:
                        results[sl.req.rid] = sl.ch.get_state()
                    sl.ch.close()
                    used -= sl.fp
                    done[sl.req.rid] = dict(t_admit=sl.t_admit, t_done=self.clock() - t0,
                                            latency=self.clock() - t0 - sl.req.t_arrival)
                    progressed = True
                else:
                    still.append(sl)
            active = still
            conc_samples.append(len(active))
            if not progressed:
                time.sleep(self.idle_sleep)
        wall = self.clock() - t0
        for b in batches.values():
            b.close()
        work = sum(r.points * r.nsub for r in requests)
        lat = [d["latency"] for d in done.values()]
        metrics = dict(requests=len(requests), wall_s=wall, packed=self.packed, batches_built=nbuilt,
                       mpts_substep_per_s=work / wall / 1e6,
                       step_ms_p50=_pct(step_ms, 50), step_ms_p99=_pct(step_ms, 99), steps_timed=len(step_ms),
                       request_s_p50=_pct(lat, 50), request_s_p99=_pct(lat, 99), max_concurrency=max_conc,
                       mean_concurrency=float(np.mean(conc_samples)) if conc_samples else 0.0,
                       setup_threads=self.setup_threads)
        return results, metrics


def _current_device():
    """The CUDA device of the calling thread (None without a GPU): set-up threads build
    their runs on the loop's device, not on the runtime's default for a new thread."""
    try:
        import torch
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except Exception:
        return None


def _set_device(dev):
    if dev is not None:
        import torch
        torch.cuda.set_device(dev)


def _torch_stream():
    import torch
    return torch.cuda.Stream()


def _torch_event():
    import torch
    return torch.cuda.Event(enable_timing=True)


def channel_factory(make_ic, use_graph=True, autotune=True):
    """Factory for Server: a Channel on the run's stream (graph replay on, launch shapes
    autotuned per shape), state from ``make_ic(request, y) -> dict(v, omega2, U1, U3)``
    with y the run's mesh."""

    def make(r, stream):
        ch = Channel(r.re_tau, r.Lx, r.Lz, r.Nx, r.Ny, r.Nz, r.dt, precision=r.precision,
                     stream=stream.cuda_stream)
        ch.set_graph(use_graph)
        s0 = make_ic(r, ch.grid())
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        if autotune:
            ch.autotune()
        return ch

    return make
