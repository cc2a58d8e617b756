"""Continuous batching of single-environment MPC solves over the C ABI.

Requests (one environment each, with the stage data of its next MPC step)
arrive over time and queue first-in first-out.  Whenever one of the
server's handles is idle and requests are waiting, the dispatcher takes up
to ``B_max`` of them, gathers their stage data into that handle's device
input buffers (on the handle's stream), and enqueues set_stages / solve /
get_traj there; a CUDA event marks the batch done.  Several handles keep
several batches in flight, so a batch forms while others run.  Each
request's latency runs from its arrival to the host observing its batch's
event.  Requests are kept in arrays and batches are formed with vectorized
index operations, so the host loop costs per batch, not per request.  With
`early` (the default), a request is answered when the round that certifies
its instance ends, not when its whole batch does: the library records an
event after each round (mpc_set_round_events), a side stream copies the
batch's statuses after it, and the requests whose status is final by then
are retired; the batch's last event retires the rest.

Every instance of a batch is solved independently, so a request's result
does not depend on which other requests share its batch (the tests check
this bit for bit).  Without `warm_shift` every request starts cold.  With
it, the server keeps each environment's solver state in a device store
(mpc_save_state / mpc_load_state): a request of an environment solved
before starts from its last state moved `warm_shift` stages (1 when each
request is the environment's next MPC step), environments with a state
are placed first in their batch, and `reset(envs)` makes the next request
of those environments cold (a new episode).  Two requests of one
environment in the same batch both start from its state before the batch.
A request whose environment is in a batch still in flight waits in the
queue (keeping its place) until that batch retires and its state is saved,
so an environment's requests see its states in request order whichever
handles serve them; the others go ahead.  With a device-memory budget the store
may hold fewer rows than environments; rows are then reclaimed least
recently used, never while a batch in flight uses them, and an environment
whose row was reclaimed starts cold.
"""
from __future__ import annotations

import time
from typing import Callable, Dict, Optional

import numpy as np

from . import pinmpc

STAGE_KEYS = ("A", "Bm", "e", "Q", "R", "ry", "ru", "mu", "fmax", "mask", "xi0", "u_prev", "horizon")
ALLOC_ROUND = 512  # the device allocator's granule: every tensor is counted rounded up to it


def _rounded(nbytes: int) -> int:
    return -(-int(nbytes) // ALLOC_ROUND) * ALLOC_ROUND


def handle_bytes(workspace: int, B_max: int, N: int, nx: int, nu: int, env_input_bytes: Dict[str, int]) -> int:
    """Device bytes of one server handle: the library workspace, the gathered
    stage-data buffers (B_max rows of every stage array), the outputs
    (u, xi, status, kkt) and the index vectors of a batch."""
    b = workspace
    b += sum(_rounded(B_max * v) for v in env_input_bytes.values())
    b += _rounded(B_max * N * nu * 4) + _rounded(B_max * N * nx * 4) + 2 * _rounded(B_max * 4)
    b += _rounded(B_max * 8) + _rounded(2 * B_max * 4)  # index vectors: environments, load and save rows
    return b


def plan_memory(budget: int, n_env: int, n_handles: int, B_max: int, per_handle, state_row_bytes: int,
                warm: bool) -> dict:
    """Admission by a device-memory budget: the most handles (batches in
    flight, up to ``n_handles``) of the largest batch size (``B_max``, halved
    while needed) that fit, then as many warm-state rows as fit, up to one
    per environment.  Every slot of every batch in flight holds a row, so
    rows >= handles x batch size.  ``per_handle(B)`` gives one handle's
    bytes at batch size B.  Raises MemoryError if one handle of batch size 1
    does not fit."""
    B = max(1, int(B_max))
    while True:
        for h in range(max(1, n_handles), 0, -1):
            used = h * per_handle(B)
            rows = 0
            if warm:
                rows = int(min(n_env, max(0, budget - used - ALLOC_ROUND) // max(state_row_bytes, 1)))
                if rows < min(n_env, h * B):
                    continue
                used += _rounded(rows * state_row_bytes)
                if used > budget:
                    continue
            if used <= budget:
                return {"handles": h, "B_max": B, "warm_rows": rows, "bytes": used}
        if B == 1:
            raise MemoryError(f"one handle of batch size 1 needs {per_handle(1)} B, budget {budget} B")
        B = max(1, B // 2)


class WarmRows:
    """Rows of the device warm-state store, assigned to environments on
    demand and reclaimed least recently used first.  A row is pinned while a
    batch in flight loads or saves it and is never reclaimed then; an
    environment whose row is reclaimed starts its next request cold."""

    def __init__(self, n_env: int, rows: int):
        self.direct = rows >= n_env  # a row per environment: row e is environment e's
        self.row_of = np.full(n_env, -1, np.int64)
        self.env_of = np.full(rows, -1, np.int64)
        self.last_use = np.zeros(rows, np.int64)
        self.pins = np.zeros(rows, np.int64)
        self.clock = 0
        self.evicted = 0

    def acquire(self, envs: np.ndarray, has_state: np.ndarray) -> np.ndarray:
        """Rows for the environments of one batch (pinned); environments whose
        row had to be taken get has_state cleared."""
        if self.direct:
            return envs
        self.clock += 1
        rows = self.row_of[envs].copy()
        need = np.unique(envs[rows < 0])
        if need.size:
            free = np.flatnonzero((self.env_of < 0) & (self.pins == 0))
            if free.size < need.size:
                cand = np.flatnonzero((self.env_of >= 0) & (self.pins == 0))
                cand = cand[~np.isin(self.env_of[cand], envs)]
                take = cand[np.argsort(self.last_use[cand], kind="stable")][:need.size - free.size]
                if free.size + take.size < need.size:
                    raise RuntimeError("warm-state rows exhausted: more slots in flight than rows")
                old = self.env_of[take]
                self.row_of[old] = -1
                has_state[old] = False
                self.env_of[take] = -1
                self.evicted += take.size
                free = np.concatenate([free, take])
            got = free[:need.size]
            self.env_of[got] = need
            self.row_of[need] = got
            rows = self.row_of[envs]
        self.last_use[rows] = self.clock
        np.add.at(self.pins, rows, 1)
        return rows

    def release(self, rows: np.ndarray):
        if not self.direct:
            np.subtract.at(self.pins, rows, 1)


class BatchServer:
    """Continuous batching over ``n_handles`` solver handles.

    ``horizon_classes`` (ascending stage counts) makes each handle run its
    ADMM rounds per horizon class, for pools with ragged horizons.
    ``mem_budget`` (bytes) admits work by device memory: the number of
    handles (batches in flight, at most ``n_handles``), the batch size (at
    most ``B_max``) and the rows of the warm-state store (at most one per
    environment, reclaimed least recently used when fewer) are chosen by
    ``plan_memory`` so that every device buffer the server allocates fits the
    budget (``self.plan``); requests beyond the slots in flight queue.
    ``pool`` holds the stage data of every environment the requests refer to
    (torch tensors on the device, keyed like ``pinmpc.device_inputs``; row e
    is environment e).  ``clock`` returns seconds.  Request r (in submission
    order) has ``env[r]``, ``t_arrival[r]``, and once served ``t_done[r]``
    and ``status[r]``.
    """

    def __init__(self, pool: Dict[str, "object"], nx: int, nc: int, contact_dim: int, B_max: int, N: int,
                 n_handles: int = 2, clock: Callable[[], float] = time.perf_counter,
                 warm_shift: Optional[int] = None, early: bool = True, horizon_classes=None,
                 mem_budget: Optional[int] = None, **overrides):
        import torch
        self.torch = torch
        self.pool = pool
        self.clock = clock
        self.device = pool["A"].device
        n_env = int(pool["A"].shape[0])
        # admission by device memory: with a budget, the handles (batches in
        # flight), the batch size and the warm-state rows are sized so that
        # everything the server allocates on the device fits it; requests
        # beyond what is in flight wait in the queue, none is dropped
        self.plan = None
        warm_rows = n_env
        if mem_budget is not None:
            nu = nc * contact_dim
            env_bytes = {k: int(pool[k][0].numel() * pool[k].element_size()) for k in STAGE_KEYS}

            def per_handle(b):
                cfg_b = pinmpc.default_config(nx, nc, contact_dim, b, N, **overrides)
                return handle_bytes(pinmpc.workspace_estimate(cfg_b), b, N, nx, nu, env_bytes)

            row_bytes = 4 * pinmpc.state_floats_estimate(pinmpc.default_config(nx, nc, contact_dim, 1, N, **overrides), N)
            self.plan = plan_memory(int(mem_budget), n_env, n_handles, B_max, per_handle, row_bytes,
                                    warm_shift is not None)
            n_handles, B_max, warm_rows = self.plan["handles"], self.plan["B_max"], self.plan["warm_rows"]
            self.plan["budget"] = int(mem_budget)
        self.B_max, self.N = B_max, N
        self.handles = []
        for _ in range(n_handles):
            cfg = pinmpc.default_config(nx, nc, contact_dim, B_max, N, **overrides)
            solver = pinmpc.Solver(cfg)
            if horizon_classes:
                solver.set_horizon_classes(list(horizon_classes))
            inputs = {k: torch.empty((B_max,) + tuple(pool[k].shape[1:]), dtype=pool[k].dtype, device=self.device)
                      for k in STAGE_KEYS}
            outs = dict(u=torch.empty((B_max, N, nc * contact_dim), dtype=torch.float32, device=self.device),
                        xi=torch.empty((B_max, N, nx), dtype=torch.float32, device=self.device),
                        status=torch.empty(B_max, dtype=torch.int32, device=self.device),
                        kkt=torch.empty(B_max, dtype=torch.float32, device=self.device))
            status_host = torch.empty(B_max, dtype=torch.int32).pin_memory()
            h = dict(solver=solver, stream=torch.cuda.Stream(self.device), inputs=inputs,
                     outs=outs, status_host=status_host, busy=None, event=None, perm=None,
                     # index vectors of a batch: environments (gather), and warm-state
                     # rows to load then rows to save (-1: none), page-locked staging
                     env_pin=torch.empty(B_max, dtype=torch.int64).pin_memory(),
                     env_dev=torch.empty(B_max, dtype=torch.int64, device=self.device),
                     row_pin=torch.empty(2 * B_max, dtype=torch.int32).pin_memory(),
                     row_dev=torch.empty(2 * B_max, dtype=torch.int32, device=self.device))
            if early:
                n_rounds = len(pinmpc.round_schedule(cfg))
                side = torch.cuda.Stream(self.device)
                round_events = [torch.cuda.Event() for _ in range(n_rounds)]
                for ev in round_events:
                    ev.record(side)  # creates the event objects
                solver.set_round_events(round_events)
                h.update(side=side, round_events=round_events,
                         round_status=[torch.empty(B_max, dtype=torch.int32).pin_memory() for _ in range(n_rounds)],
                         round_copied=[torch.cuda.Event() for _ in range(n_rounds)], next_round=0, answered=None)
            self.handles.append(h)
        self.early = early
        self.warm_shift = warm_shift
        self.warm_loads = 0
        if warm_shift is not None:
            rows = self.handles[0]["solver"].state_floats(N)
            self.store = torch.zeros((warm_rows, rows), dtype=torch.float32, device=self.device)
            self.has_state = np.zeros(n_env, dtype=bool)
            self.rows = WarmRows(n_env, warm_rows)
            self.slot_of = np.zeros(n_env, np.int64)  # scratch: an environment's last slot in a batch
        cap = 1 << 16
        self.env = np.zeros(cap, np.int64)
        self.t_arrival = np.zeros(cap)
        self.t_done = np.full(cap, np.nan)
        self.status = np.full(cap, -1, np.int32)
        self.n = 0          # requests submitted
        self.head = 0       # first request not yet looked at by the dispatcher
        # requests passed over because their environment's previous batch was
        # still in flight (its saved state not yet final), oldest first
        self.deferred = np.zeros(0, np.int64)
        self.batches = 0
        if warm_shift is not None:
            # the batch (serial number) that last took each environment, while in flight
            self.env_batch = np.full(n_env, -1, np.int64)
            self.deferrals = 0
        self.results: Dict[int, dict] = {}
        self.keep_results = False

    def _grow(self, need):
        cap = len(self.env)
        while cap < need:
            cap *= 2
        if cap != len(self.env):
            for name, fill in (("env", 0), ("t_arrival", 0.0), ("t_done", np.nan), ("status", -1)):
                a = getattr(self, name)
                b = np.full(cap, fill, a.dtype)
                b[:len(a)] = a
                setattr(self, name, b)

    def submit(self, envs, t_arrival: Optional[np.ndarray] = None):
        """Queue requests for environments `envs` (arrival times default to now)."""
        envs = np.atleast_1d(np.asarray(envs, np.int64))
        k = len(envs)
        self._grow(self.n + k)
        self.env[self.n:self.n + k] = envs
        self.t_arrival[self.n:self.n + k] = self.clock() if t_arrival is None else t_arrival
        self.n += k

    @property
    def queued(self) -> int:
        return self.n - self.head + len(self.deferred)

    def busy(self) -> bool:
        return any(h["busy"] is not None for h in self.handles)

    def reset(self, envs):
        """The next request of each of `envs` starts cold (a new episode)."""
        if self.warm_shift is not None:
            self.has_state[np.atleast_1d(np.asarray(envs, np.int64))] = False

    def _take(self) -> np.ndarray:
        """Request ids of the next batch, first-in first-out among those that
        may go: with warm state, a request whose environment is in a batch
        still in flight waits (its state is saved when that batch ends) and
        keeps its place ahead of later requests."""
        if self.warm_shift is None:
            lo = self.head
            self.head = min(self.n, lo + self.B_max)
            return np.arange(lo, self.head)
        free = self.env_batch < 0
        d_ok = free[self.env[self.deferred]]
        take = self.deferred[d_ok][:self.B_max]
        kept = np.concatenate([self.deferred[d_ok][self.B_max:], self.deferred[~d_ok]])
        need = self.B_max - len(take)
        parts, wait = [take], [kept]
        while need > 0 and self.head < self.n:
            chunk = np.arange(self.head, min(self.n, self.head + 2 * need))
            ok = free[self.env[chunk]]
            pos = np.flatnonzero(ok)
            if len(pos) > need:  # stop after the need-th eligible request
                chunk, ok = chunk[:pos[need - 1] + 1], ok[:pos[need - 1] + 1]
            parts.append(chunk[ok])
            wait.append(chunk[~ok])
            self.head = int(chunk[-1]) + 1
            need -= int(ok.sum())
        out = np.concatenate(parts)
        self.deferred = np.sort(np.concatenate(wait))
        self.deferrals += sum(len(w) for w in wait[1:])
        return out

    def _dispatch(self, h):
        torch = self.torch
        reqs = self._take()
        B = len(reqs)
        if B == 0:
            return
        envs = self.env[reqs]
        perm = None
        n_warm = 0
        if self.warm_shift is not None:
            # environments with a saved state first (slots [0, n_warm))
            warm = self.has_state[envs]
            perm = np.argsort(~warm, kind="stable")
            envs = envs[perm]
            n_warm = int(warm.sum())
        rows = None
        # the batch's index vectors go up in one asynchronous copy from this
        # handle's page-locked staging (free again: the handle's last batch
        # has retired), before anything of the batch is enqueued -- a copy from
        # pageable memory would block the host until the stream reached it
        h["env_pin"][:B] = torch.from_numpy(envs)
        if self.warm_shift is not None:
            rows = self.rows.acquire(envs, self.has_state)  # pinned until the batch retires
            # one writer per row: an environment with several requests in the
            # batch saves from its last slot only
            slots = np.arange(B)
            self.slot_of[envs] = slots  # repeated environments: the last slot's write stays
            save = np.where(self.slot_of[envs] == slots, rows, -1)
            h["row_pin"][:B] = torch.from_numpy(rows.astype(np.int32))
            h["row_pin"][self.B_max:self.B_max + B] = torch.from_numpy(save.astype(np.int32))
        with torch.cuda.stream(h["stream"]):
            h["env_dev"][:B].copy_(h["env_pin"][:B], non_blocking=True)
            if self.warm_shift is not None:
                h["row_dev"].copy_(h["row_pin"], non_blocking=True)
            idx64 = h["env_dev"][:B]
            for k in STAGE_KEYS:
                torch.index_select(self.pool[k], 0, idx64, out=h["inputs"][k][:B])
        view = {k: h["inputs"][k][:B] for k in STAGE_KEYS}
        s = h["solver"]
        s.set_stages(B, self.N, **view, stream=h["stream"])
        if self.warm_shift is not None:
            ridx = h["row_dev"][:B]
            sidx = h["row_dev"][self.B_max:self.B_max + B]
        if n_warm:
            # every row was last saved by a batch that has retired (its
            # environment waited in the queue for that), so no device wait is needed
            s.load_state(self.store, ridx, n_warm, stream=h["stream"])
            self.warm_loads += n_warm
        s.solve(B, stream=h["stream"])
        if self.warm_shift is not None:
            s.save_state(self.store, sidx, B, shift=self.warm_shift, stream=h["stream"])
            self.has_state[envs] = True
            self.env_batch[envs] = self.batches
        h["rows"] = rows
        o = h["outs"]
        if self.early:
            # after each round: that round's statuses into pinned memory on the side stream
            for r, ev in enumerate(h["round_events"]):
                h["side"].wait_event(ev)
                s.get_traj(status=h["round_status"][r], stream=h["side"])
                h["round_copied"][r].record(h["side"])
            h["next_round"] = 0
            h["answered"] = np.zeros(B, dtype=bool)
        s.get_traj(xi=o["xi"], u=o["u"], status=o["status"], kkt=o["kkt"], stream=h["stream"])
        with torch.cuda.stream(h["stream"]):
            h["status_host"][:B].copy_(o["status"][:B], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(h["stream"])
        h["busy"], h["event"], h["perm"] = reqs, ev, perm
        h["serial"] = self.batches
        self.batches += 1

    def _answer_early(self, h, now):
        """Retire the requests whose instances the rounds copied so far finished."""
        reqs = h["busy"]
        # slot i holds request reqs[order[i]]
        order = reqs[h["perm"]] if h["perm"] is not None else reqs
        while h["next_round"] < len(h["round_events"]) and h["round_copied"][h["next_round"]].query():
            st = h["round_status"][h["next_round"]][:len(reqs)].numpy()
            new = (st != pinmpc.RUNNING) & ~h["answered"]
            if new.any():
                now = self.clock() if now is None else now
                req = order[new]
                self.t_done[req] = now
                self.status[req] = st[new]
                h["answered"] |= new
            h["next_round"] += 1
        return now

    def _retire(self, h, now):
        reqs = h["busy"]
        B = len(reqs)
        # slot i holds request order[i]
        order = reqs[h["perm"]] if h["perm"] is not None else reqs
        late = ~h["answered"] if self.early else np.ones(B, dtype=bool)
        self.t_done[order[late]] = now
        self.status[order] = h["status_host"][:B].numpy()
        if self.keep_results:
            o = {k: h["outs"][k][:B].cpu().numpy() for k in ("u", "xi", "kkt")}
            for i in range(B):
                self.results[int(order[i])] = {k: o[k][i] for k in o}
        if h.get("rows") is not None:
            self.rows.release(h["rows"])
            h["rows"] = None
        if self.warm_shift is not None:
            # its environments may go again (their states are saved)
            envs = self.env[reqs]
            mine = self.env_batch[envs] == h["serial"]
            self.env_batch[envs[mine]] = -1
        h["busy"], h["event"], h["perm"] = None, None, None

    def step(self):
        """One pass of the serving loop: retire finished batches, start new ones."""
        now = None
        for h in self.handles:
            if h["busy"] is None:
                continue
            if self.early:
                now = self._answer_early(h, now)
                if h["next_round"] < len(h["round_events"]):
                    continue  # the side stream still copies this batch's statuses
            if h["event"].query():
                now = self.clock() if now is None else now
                self._retire(h, now)
        for h in self.handles:
            if h["busy"] is None and self.queued:
                self._dispatch(h)

    def drain(self):
        while self.queued or self.busy():
            self.step()

    def close(self):
        for h in self.handles:
            h["solver"].close()


def poisson_arrivals(rate: float, duration: float, n_env: int, seed: int = 0) -> np.ndarray:
    """[(t, env)] with exponential inter-arrival times (rate per second) over
    `duration` seconds, environments drawn uniformly."""
    rng = np.random.default_rng(seed)
    n = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    t = t[t < duration]
    env = rng.integers(0, n_env, size=t.size)
    return np.stack([t, env], axis=1)


def serve_load(server: BatchServer, arrivals: np.ndarray) -> dict:
    """Replay `arrivals` in real time through `server`; per-request latency
    percentiles (ms) and the achieved throughput (requests/s)."""
    t0 = server.clock()
    i, n = 0, len(arrivals)
    first, batches0 = server.n, server.batches
    times = arrivals[:, 0]
    while i < n or server.queued or server.busy():
        now = server.clock() - t0
        j = int(np.searchsorted(times, now, side="right"))
        if j > i:
            server.submit(arrivals[i:j, 1].astype(np.int64), t0 + times[i:j])
            i = j
        server.step()
    lo, hi = first, server.n
    lat = (server.t_done[lo:hi] - server.t_arrival[lo:hi]) * 1e3
    span = float(np.max(server.t_done[lo:hi])) - t0
    return {"requests": hi - lo, "certified": int(np.sum(server.status[lo:hi] == 0)),
            "offered_per_s": (hi - lo) / max(float(times[-1]), 1e-9), "achieved_per_s": (hi - lo) / span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batch": (hi - lo) / max(server.batches - batches0, 1)}


def fleet_load(server, hz: float = 50.0, duration: float = 1.0, warmup: float = 0.0, reset_rate: float = 0.0,
               seed: int = 0) -> dict:
    """A fleet of controllers, one per environment of the server's pool, each
    ticking at `hz` (phases uniform).  At each tick an environment requests
    the solve of its next MPC step, unless its previous request is still
    unanswered: then the tick is counted as skipped (the controller keeps its
    last plan) -- nothing is dropped silently.  Episodes end as a Poisson
    process of `reset_rate` per environment per second; `server.reset(env)`
    makes the environment's next request cold.

    Runs for `warmup` + `duration` seconds of the server's clock, then drains.
    Figures cover the measured window [warmup, warmup + duration): ticks,
    requests submitted, skipped ticks, requests answered in the window per
    second, and the latency percentiles (tick to answer) of the requests
    that arrived in it."""
    n_env = int(server.pool["A"].shape[0])
    rng = np.random.default_rng(seed)
    period = 1.0 / hz
    next_tick = rng.uniform(0.0, period, n_env)
    next_reset = rng.exponential(1.0 / reset_rate, n_env) if reset_rate > 0 else np.full(n_env, np.inf)
    pending = np.full(n_env, -1, np.int64)
    end = warmup + duration
    counts = dict(ticks=0, skipped=0, resets=0)
    t0 = server.clock()
    first = server.n
    while True:
        now = server.clock() - t0
        if now >= end:
            break
        measured = now >= warmup
        due_r = next_reset <= now
        if due_r.any():
            er = np.flatnonzero(due_r)
            server.reset(er)
            if measured:
                counts["resets"] += er.size
            next_reset[er] += rng.exponential(1.0 / reset_rate, er.size)
        busy = np.flatnonzero(pending >= 0)
        if busy.size:
            answered = ~np.isnan(server.t_done[pending[busy]])
            pending[busy[answered]] = -1
        idx = np.flatnonzero(next_tick <= now)
        if idx.size:
            nt = np.floor((now - next_tick[idx]) / period).astype(np.int64) + 1  # ticks passed since the last look
            free = pending[idx] < 0
            sub = idx[free]
            if measured:
                counts["ticks"] += int(nt.sum())
                counts["skipped"] += int(nt.sum()) - sub.size
            if sub.size:
                # each request arrives at its environment's latest tick
                t_arr = t0 + next_tick[sub] + (nt[free] - 1) * period
                pending[sub] = np.arange(server.n, server.n + sub.size)
                server.submit(sub, t_arr)
            next_tick[idx] += nt * period
        server.step()
    server.drain()
    lo, hi = first, server.n
    t_arr = server.t_arrival[lo:hi] - t0
    t_done = server.t_done[lo:hi] - t0
    win = (t_arr >= warmup) & (t_arr < end)
    lat = (t_done[win] - t_arr[win]) * 1e3
    done_in = int(np.sum((t_done >= warmup) & (t_done < end)))
    return {"envs": n_env, "hz": hz, "window_s": duration,
            "offered_ticks_per_s": counts["ticks"] / duration,
            "requests": int(win.sum()), "skipped_ticks": counts["skipped"], "resets": counts["resets"],
            "answered_per_s": done_in / duration,
            "deferred": int(getattr(server, "deferrals", 0)),
            "certified": int(np.sum(server.status[lo:hi][win] == 0)),
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None}
