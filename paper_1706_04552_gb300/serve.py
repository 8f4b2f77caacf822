"""Continuous-batching server for CA-step requests on resident gaskets.

Requests ask for k steps of the gasket-restricted B3/S23 automaton on one
of many resident gaskets of different levels.  The serving loop:

  * admits requests as they arrive (their arrival times are real time on
    the host clock) into per-gasket FIFOs;
  * keeps every gasket's state on the device while it fits a device-memory
    budget; a gasket that does not fit is brought in from pinned host memory
    after evicting the least recently used idle gaskets (their current state
    goes back to pinned host memory);
  * runs iterations: every gasket whose head request still has steps left
    advances one step, all of them in ONE batched launch (a prefix-summed
    work list over the active gaskets' lambda block spaces, sg_batch_ca_*),
    so requests that arrive while others are on the GPU join at the next
    iteration; a request completes when its last step has run;
  * reports per-request latency (arrival to completion) and throughput.

With fuse > 1 an iteration advances a gasket by up to `fuse` steps at once:
the active gaskets are grouped by the largest power of two k <= min(fuse,
steps left in the head request), and each group is one batched launch of k
fused steps (sg_batch_ca_steps).  A gasket never steps past its head
request, so every result is still the plain per-gasket step sequence.

mode="per_gasket" runs the same scheduler with one single-gasket launch per
active gasket per iteration instead of the batched launch, for comparison.

Two engines run the batched mode.  engine="native" hands the queues and the
iteration to the C++ core (include/sg_sched.h): Python admits arrivals in
slices, keeps residency (loads and evictions) and stamps completions, and
each iteration's grouping, work lists and launches are built natively.  The
core advances a gasket by min(fuse, steps left in its head request) in one
launch rather than by a power of two: gaskets whose advances stage the same
halo (1 step; 2..4; 5..8; 9..16) share a launch, each running its own count,
so a request of 7 steps takes one launch instead of three.  Its
work lists reach the device by an asynchronous copy from page-locked memory,
so up to `pipeline` iterations are in flight: the host prepares the next one
while the device runs the current one, and a request's completion is stamped
when the host sees its iteration's event complete.  engine="python" is the
same policy written out in Python, one iteration at a time (and the one the
per-gasket comparison uses).

Failures are contained on the host.  A launch that the library refuses
(an SGError from its C ABI) fails the head requests of the gaskets it was
for: nothing ran, their states stay as they were, and the rest of the
iteration and of the trace go on.  A gasket that cannot be brought onto the
device fails the requests queued for it and stays in host memory.  Each
failure is recorded with its error and the steps of the request that had
already run; a failed request's steps that ran stay applied.

Every gasket's state follows the plain per-gasket sequence of CA steps in
arrival order of its requests, so each result equals stepping the gasket
alone; tests check that against single-gasket runs and the CPU oracle.
"""
from __future__ import annotations

import ctypes
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class ServeConfig:
    gaskets: int = 500
    level_min: int = 6
    level_max: int = 15
    level_decay: float = 0.5          # P(level = min + k) proportional to decay^k
    rate: float = 2000.0              # mean arrivals per second (Poisson)
    steps_min: int = 1
    steps_max: int = 32
    duration: float = 2.0             # seconds of arrivals
    budget_bytes: int = 40 << 30      # device bytes for resident gasket states
    seed: int = 3
    ca_p: float = 0.3
    rho: int = 64
    mode: str = "batched"             # or "per_gasket"
    fuse: int = 1                     # most steps one iteration advances a gasket (batched)
    engine: str = "native"            # batched mode: "native" (sg_sched) or "python"
    pipeline: int = 2                 # native: iterations in flight on the stream


def gasket_levels(cfg: ServeConfig) -> np.ndarray:
    """Levels drawn geometrically toward small levels (seeded)."""
    ks = np.arange(cfg.level_max - cfg.level_min + 1)
    p = cfg.level_decay ** ks
    p /= p.sum()
    rng = np.random.default_rng(cfg.seed)
    return cfg.level_min + rng.choice(len(ks), size=cfg.gaskets, p=p)


def make_trace(cfg: ServeConfig):
    """Poisson arrivals over cfg.duration: (arrival s, gasket id, steps)."""
    rng = np.random.default_rng(cfg.seed + 1)
    n = int(rng.poisson(cfg.rate * cfg.duration))
    t = np.sort(rng.uniform(0.0, cfg.duration, n))
    g = rng.integers(0, cfg.gaskets, n)
    k = rng.integers(cfg.steps_min, cfg.steps_max + 1, n)
    return t, g, k


def launch_groups(fuse: int) -> list[int]:
    """Step counts of the launch groups an iteration may use: 1, 2, 4, ...
    up to fuse."""
    return [1 << j for j in range(int(fuse).bit_length()) if (1 << j) <= fuse]


def steps_this_iteration(left: int, groups: list[int]) -> int:
    """Steps a gasket whose head request has `left` steps to go advances in
    one iteration: the largest group size not above `left`."""
    return max(k for k in groups if k <= left)


class _Gasket:
    __slots__ = ("gid", "level", "n2", "host", "cur", "nxt", "resident", "queue",
                 "last_use", "steps_done", "advance")

    def __init__(self, gid, level, host):
        self.gid = gid
        self.level = int(level)
        self.n2 = 1 << (2 * self.level)
        self.host = host                  # pinned host copy (current state when evicted)
        self.cur = self.nxt = None        # device buffers while resident
        self.resident = False
        self.queue = []                   # [request index, steps left] in arrival order
        self.last_use = 0
        self.steps_done = 0
        self.advance = 1                  # steps the current iteration takes

    @property
    def device_bytes(self):
        return 2 * self.n2


class Server:
    """The serving loop over one CUDA stream (see the module docstring)."""

    def __init__(self, cfg: ServeConfig, initial_states=None, device="cuda"):
        import torch
        import paper_1706_04552_gb300 as sg
        from paper_1706_04552_gb300 import inputs
        self.torch, self.sg, self.cfg = torch, sg, cfg
        self.dev = torch.device(device)
        self.stream = torch.cuda.current_stream(self.dev)
        levels = gasket_levels(cfg)
        self.gaskets = []
        for i, r in enumerate(levels):
            host = torch.empty(1 << (2 * int(r)), dtype=torch.uint8, pin_memory=True)
            if initial_states is not None:
                host.copy_(torch.from_numpy(initial_states[i].ravel()))
            else:
                idx, vals = inputs.ca_seed_sparse(int(r), cfg.ca_p, inputs.instance_seed(cfg.seed, i))
                host.zero_()
                host[torch.from_numpy(idx)] = torch.from_numpy(vals)
            self.gaskets.append(_Gasket(i, r, host))
        self.used = 0
        self.evictions = 0
        self.loads = 0
        self.failures = []                # per failed request: (request, gasket, steps run, error)
        cnt = len(self.gaskets)
        if cfg.fuse < 1 or cfg.fuse > sg.FUSE_MAX:
            raise ValueError(f"fuse must be 1..{sg.FUSE_MAX}")
        # one work-list workspace per launch group (k = 1, 2, 4, ...)
        self.ks = launch_groups(cfg.fuse)
        wsb = int(sg.lib().sg_batch_workspace_bytes(cnt))
        self.ws = [torch.empty(wsb, dtype=torch.uint8, device=self.dev) for _ in self.ks]
        self._lv = np.zeros(cnt, dtype=np.int32)
        self._pa = np.zeros(cnt, dtype=np.uint64)
        self._pb = np.zeros(cnt, dtype=np.uint64)
        self._plan = sg.BatchPlan()
        if cfg.engine not in ("native", "python"):
            raise ValueError("engine must be 'native' or 'python'")
        if cfg.pipeline < 1:
            raise ValueError("pipeline must be >= 1")
        self.native = cfg.mode == "batched" and cfg.engine == "native"
        self.sched = sg.Sched(levels, cfg.rho, cfg.fuse) if self.native else None
        self.tick = 0
        self._preload()
        self._warm_up()

    def _preload(self):
        """Bring gaskets onto the device, in order, while they fit the budget:
        the resident state a server starts from (the rest load on demand)."""
        for g in self.gaskets:
            if self.used + g.device_bytes > self.cfg.budget_bytes:
                break
            self._make_resident(g, set())
        self.loads = 0
        self.stream.synchronize()

    def _warm_up(self):
        """Launch every kernel the loop will use once, on a scratch gasket of
        all-dead cells, so that the first requests do not pay for loading
        kernels or for occupancy queries."""
        torch, sg = self.torch, self.sg
        r = max(6, self.cfg.rho.bit_length() - 1)
        a = torch.zeros(1 << (2 * r), dtype=torch.uint8, device=self.dev)
        b = torch.zeros_like(a)
        if self.cfg.mode == "per_gasket":
            sg.ca_step(a, b, r, self.cfg.rho, "lambda", self.stream)
        else:
            L = sg.lib()
            lv = np.array([r], dtype=np.int32)
            pa = np.array([a.data_ptr()], dtype=np.uint64)
            pb = np.array([b.data_ptr()], dtype=np.uint64)
            for slot, k in enumerate(self.ks):
                ws = self.ws[slot]
                sg._check("sg_batch_ca_plan", int(L.sg_batch_ca_plan(
                    1, lv.ctypes.data, pa.ctypes.data, pb.ctypes.data, self.cfg.rho,
                    ws.data_ptr(), ws.numel(), ctypes.byref(self._plan), self.stream.cuda_stream)))
                sg._check("sg_batch_ca_steps", int(L.sg_batch_ca_steps(
                    ctypes.byref(self._plan), 0, k, None, self.stream.cuda_stream)))
        self.stream.synchronize()

    # ------------------------------------------------------------ residency
    def _idle(self, g):
        return (self.sched.gasket(g.gid).queued == 0) if self.native else not g.queue

    def _last_use(self, g):
        return int(self.sched.gasket(g.gid).last_use) if self.native else g.last_use

    def _sync_bufs(self, g):
        """Native engine: point g.cur at the buffer the scheduler holds as
        current (it swaps the two after every iteration that advances g)."""
        if self.native and g.resident and self.sched.gasket(g.gid).cur != g.cur.data_ptr():
            g.cur, g.nxt = g.nxt, g.cur

    def _evict_one(self, protect):
        idle = [g for g in self.gaskets if g.resident and g.gid not in protect and self._idle(g)]
        if not idle:
            return False
        v = min(idle, key=self._last_use)
        self._sync_bufs(v)
        v.host.copy_(v.cur, non_blocking=True)           # current state back to host
        self.stream.synchronize()
        if self.native:
            self.sched.set_buffers(v.gid, 0, 0)
        v.cur = v.nxt = None
        v.resident = False
        self.used -= v.device_bytes
        self.evictions += 1
        return True

    def _make_resident(self, g, protect):
        if g.resident:
            return True
        while self.used + g.device_bytes > self.cfg.budget_bytes:
            if not self._evict_one(protect):
                return False
        torch = self.torch
        g.cur = torch.empty(g.n2, dtype=torch.uint8, device=self.dev)
        g.nxt = torch.zeros(g.n2, dtype=torch.uint8, device=self.dev)
        g.cur.copy_(g.host, non_blocking=True)
        g.resident = True
        if self.native:
            self.sched.set_buffers(g.gid, g.cur.data_ptr(), g.nxt.data_ptr())
        self.used += g.device_bytes
        self.loads += 1
        return True

    # ------------------------------------------------------------- stepping
    def _steps_for(self, g):
        return steps_this_iteration(g.queue[0][1], self.ks)

    def _launch(self, group, k):
        """One launch of k steps for `group` (one gasket in per-gasket mode).
        Raises SGError when the library refuses it; nothing has run then."""
        sg = self.sg
        if self.cfg.mode == "per_gasket":
            g = group[0]
            sg.ca_step(g.cur, g.nxt, g.level, min(self.cfg.rho, 1 << g.level), "lambda",
                       self.stream)
            return
        L = sg.lib()
        for j, g in enumerate(group):
            self._lv[j] = g.level
            self._pa[j] = g.cur.data_ptr()
            self._pb[j] = g.nxt.data_ptr()
        ws = self.ws[self.ks.index(k)]
        st = L.sg_batch_ca_plan(len(group), self._lv.ctypes.data, self._pa.ctypes.data,
                                self._pb.ctypes.data, self.cfg.rho, ws.data_ptr(), ws.numel(),
                                ctypes.byref(self._plan), self.stream.cuda_stream)
        sg._check("sg_batch_ca_plan", int(st))
        sg._check("sg_batch_ca_steps", int(L.sg_batch_ca_steps(
            ctypes.byref(self._plan), 0, k, None, self.stream.cuda_stream)))

    def _step(self, active):
        """Advance every active gasket.  Returns (launches, gaskets whose
        launch was refused, with the error)."""
        failed = {}
        if self.cfg.mode == "per_gasket":
            groups = [([g], 1) for g in active]
        else:
            groups = [([g for g in active if g.advance == k], k) for k in self.ks]
        launches = 0
        for group, k in groups:
            if not group:
                continue
            try:
                self._launch(group, k)
                launches += 1
            except self.sg.SGError as e:
                for g in group:
                    failed[g.gid] = str(e)
        return launches, failed

    # ----------------------------------------------------------------- loop
    def run(self, trace, on_complete=None):
        """Serve a trace (arrival s, gasket, steps).  on_complete(req, gasket)
        is called right after a request's last step (state in gasket.cur).
        Returns per-request arrival/completion times, which requests failed,
        and counters.  busy_s is device time: CUDA events around every
        iteration's work on the serving stream."""
        if self.native:
            return self._run_native(trace, on_complete)
        torch = self.torch
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t_arr, g_id, k_steps = trace
        nreq = len(t_arr)
        done_at = np.full(nreq, np.nan)
        start_at = np.full(nreq, np.nan)
        failed = np.zeros(nreq, dtype=bool)
        busy = 0.0
        iters = 0
        launches = 0
        cells = 0
        nxt = 0
        remaining = nreq
        pending = {}                      # gasket id -> gasket, for gaskets with requests
        t0 = time.perf_counter()
        while remaining:
            now = time.perf_counter() - t0
            while nxt < nreq and t_arr[nxt] <= now:
                g = self.gaskets[int(g_id[nxt])]
                g.queue.append([nxt, int(k_steps[nxt])])
                pending[g.gid] = g
                nxt += 1
            if not pending:
                if nxt < nreq:
                    dt = t_arr[nxt] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(min(dt, 0.0001))
                continue
            waiting = list(pending.values())
            protect = set(pending)
            active = []
            for g in waiting:
                try:
                    ok = self._make_resident(g, protect)
                except Exception as e:          # the copy in failed: its requests fail
                    now = time.perf_counter() - t0
                    while g.queue:
                        req, left = g.queue.pop(0)
                        self.failures.append((req, g.gid, int(k_steps[req]) - left, str(e)))
                        failed[req] = True
                        done_at[req] = now
                        remaining -= 1
                    del pending[g.gid]
                    continue
                if ok:
                    active.append(g)
            if not active:
                if pending:
                    raise RuntimeError("a requested gasket does not fit the device budget")
                continue
            self.tick += 1
            for g in active:
                g.advance = self._steps_for(g) if self.cfg.mode == "batched" else 1
            tb = time.perf_counter()
            ev0.record(self.stream)
            n_launch, refused = self._step(active)
            ev1.record(self.stream)
            launches += n_launch
            self.stream.synchronize()
            te = time.perf_counter()
            busy += ev0.elapsed_time(ev1) / 1e3
            iters += 1
            tdone = te - t0
            for g in active:
                if g.gid in refused:           # nothing ran: its head request fails
                    req, left = g.queue.pop(0)
                    self.failures.append((req, g.gid, int(k_steps[req]) - left, refused[g.gid]))
                    failed[req] = True
                    done_at[req] = tdone
                    remaining -= 1
                    g.last_use = self.tick
                    if not g.queue:
                        del pending[g.gid]
                    continue
                g.cur, g.nxt = g.nxt, g.cur
                g.last_use = self.tick
                g.steps_done += g.advance
                cells += 3 ** g.level * g.advance
                head = g.queue[0]
                if np.isnan(start_at[head[0]]):
                    start_at[head[0]] = tb - t0
                head[1] -= g.advance
                if head[1] == 0:
                    g.queue.pop(0)
                    done_at[head[0]] = tdone
                    remaining -= 1
                    if not g.queue:
                        del pending[g.gid]
                    if on_complete is not None:
                        on_complete(head[0], g)
        wall = time.perf_counter() - t0
        lat = done_at - t_arr
        return {"requests": nreq, "wall_s": wall, "iterations": iters, "launches": launches,
                "busy_s": busy, "cell_steps": cells, "latency_s": lat, "arrival_s": t_arr,
                "failed": failed, "evictions": self.evictions, "loads": self.loads}

    def _run_native(self, trace, on_complete):
        """run() on the native core (sg_sched): admission in slices, up to
        cfg.pipeline iterations in flight, completions stamped when their
        iteration's event is seen complete."""
        import collections
        torch, sched, sg = self.torch, self.sched, self.sg
        t_arr, g_id, k_steps = trace
        nreq = len(t_arr)
        t_arr = np.asarray(t_arr, dtype=np.float64)
        gid32 = np.ascontiguousarray(g_id, dtype=np.int32)
        k32 = np.ascontiguousarray(k_steps, dtype=np.int32)
        ids = np.arange(nreq, dtype=np.int64)
        done_at = np.full(nreq, np.nan)
        failed = np.zeros(nreq, dtype=bool)
        depth = int(self.cfg.pipeline)
        # one pair of events per iteration in flight, reused round robin
        ring = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(depth)]
        inflight = collections.deque()         # (events, requests it completes)
        busy = 0.0
        iters = launches = cells = 0
        nxt = 0
        remaining = nreq
        t0 = time.perf_counter()

        def retire(block):
            # stamp the iterations that have finished (the oldest one waited
            # for when block); returns how many requests that completed
            nonlocal busy, remaining
            while inflight:
                (e0, e1), done = inflight[0]
                if block:
                    e1.synchronize()
                    block = False
                elif not e1.query():
                    return
                busy += e0.elapsed_time(e1) / 1e3
                done_at[done] = time.perf_counter() - t0
                remaining -= len(done)
                inflight.popleft()

        while remaining:
            now = time.perf_counter() - t0
            if nxt < nreq:
                j = int(np.searchsorted(t_arr, now, side="right"))
                if j > nxt:
                    sched.submit(gid32[nxt:j], ids[nxt:j], k32[nxt:j])
                    nxt = j
            unfit = False
            for g in sched.waiting().tolist():
                gg = self.gaskets[g]
                try:
                    ok = self._make_resident(gg, set())
                except Exception as e:          # the copy in failed: its requests fail
                    req, ran = sched.drop(g)
                    tnow = time.perf_counter() - t0
                    for rq, kr in zip(req.tolist(), ran.tolist()):
                        self.failures.append((rq, g, kr, str(e)))
                    failed[req] = True
                    done_at[req] = tnow
                    remaining -= len(req)
                    continue
                unfit |= not ok
            if len(inflight) >= depth:
                retire(True)
            e0, e1 = ring[iters % depth]
            e0.record(self.stream)
            res = sched.step(self.stream)
            if res.iteration == 0:              # nothing resident to advance
                retire(False)
                if unfit and not inflight:
                    raise RuntimeError("a requested gasket does not fit the device budget")
                if not inflight and nxt < nreq:
                    dt = t_arr[nxt] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(min(dt, 0.0001))
                continue
            e1.record(self.stream)
            iters += 1
            launches += int(res.launches)
            cells += int(res.cell_steps)
            done, done_g = sched.completed()
            done = done.copy()
            if res.n_failed:                    # launches refused: nothing ran for them
                freq, fg, fran = sched.failed()
                err = "batched launch refused: " + sg.lib().sg_last_error_string().decode()
                tnow = time.perf_counter() - t0
                for rq, g, kr in zip(freq.tolist(), fg.tolist(), fran.tolist()):
                    self.failures.append((rq, g, kr, err))
                failed[freq] = True
                done_at[freq] = tnow
                remaining -= int(res.n_failed)
            if on_complete is not None:
                for rq, g in zip(done.tolist(), done_g.tolist()):
                    gg = self.gaskets[g]
                    self._sync_bufs(gg)
                    on_complete(rq, gg)
            inflight.append(((e0, e1), done))
            retire(False)
        wall = time.perf_counter() - t0
        for g in self.gaskets:
            self._sync_bufs(g)
        lat = done_at - t_arr
        return {"requests": nreq, "wall_s": wall, "iterations": iters, "launches": launches,
                "busy_s": busy, "cell_steps": cells, "latency_s": lat, "arrival_s": t_arr,
                "failed": failed, "evictions": self.evictions, "loads": self.loads}

    def state_of(self, gid):
        """Current state of gasket gid (host numpy copy)."""
        g = self.gaskets[gid]
        n = 1 << g.level
        self._sync_bufs(g)
        src = g.cur if g.resident else g.host
        self.stream.synchronize()
        return src.cpu().numpy().reshape(n, n)


def summarize(res, cfg: ServeConfig):
    lat_ms = res["latency_s"] * 1e3
    return {
        "mode": cfg.mode if cfg.fuse == 1 else f"{cfg.mode}, up to {cfg.fuse} fused steps",
        "requests": int(res["requests"]),
        "failed": int(res["failed"].sum()),
        "offered_rate_rps": cfg.rate,
        "throughput_rps": round(res["requests"] / res["wall_s"], 1),
        "cell_steps_per_s_G": round(res["cell_steps"] / res["wall_s"] / 1e9, 4),
        "gpu_busy_fraction": round(res["busy_s"] / res["wall_s"], 4),
        "latency_ms_p50": round(float(np.percentile(lat_ms, 50)), 3),
        "latency_ms_p99": round(float(np.percentile(lat_ms, 99)), 3),
        "latency_ms_max": round(float(np.max(lat_ms)), 3),
        "iterations": int(res["iterations"]),
        "launches": int(res["launches"]),
        "evictions": int(res["evictions"]),
        "loads": int(res["loads"]),
        "wall_s": round(res["wall_s"], 3),
    }
