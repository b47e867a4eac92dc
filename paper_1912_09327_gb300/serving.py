"""Continuous-batching service for LBMTau1 solves.

Requests (a domain to solve to a steady-state residual) arrive over time.
The service keeps every admitted domain's fields on the device and advances
all of them together with the batched step (one launch per time step for the
whole batch, lbm_batch_step).  Between chunks of steps it reads every member's
residual with one copy, retires the converged members (their final state is
downloaded and their memory freed), and admits waiting requests while batch
slots, the device-memory budget and the active-node budget allow: new work
joins while older work is still on the device.  Waiting requests are taken
smallest first (fewest nodes), so short solves are not held behind long ones,
with a bound on how long any request waits before it goes first; the
active-node budget keeps the batch large enough to fill the GPU but not so
large that every member's steps slow down.  All arithmetic runs in the
library's kernels; this module only schedules.

The plain sequential form, `serve_sequential`, solves the same requests one at
a time in arrival order, for comparison.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    completed: float
    steps: int
    residual: float
    converged: bool
    nodes: int
    state: tuple = field(default=None, repr=False)  # float32 (rho-1, jx, jy)

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


def _footprint(req) -> int:
    p = binding.make_params(req.nx, req.ny)
    return binding.lbm_workspace_bytes(p)


def select_next(waiting, now, policy="sjf", max_wait=2.0):
    """The request to admit next: the one that arrived first under "fifo", or
    when it has waited longer than `max_wait` seconds; otherwise the one with
    the fewest nodes (earliest arrival among equals)."""
    if not waiting:
        return None
    oldest = min(waiting, key=lambda r: (r.arrival, r.rid))
    if policy == "fifo" or now - oldest.arrival > max_wait:
        return oldest
    return min(waiting, key=lambda r: (r.nx * r.ny, r.arrival, r.rid))


TWO_COLUMN_COST = 1.215  # per column, two columns per lane against four

# Active-node budget of the service: 8 Mi nodes keep a GB300's 152 SMs busy
# with several waves of block tiles; measured on the 32-request Poisson mix
# (sides 64..2048) it cuts the median latency by about a quarter against no
# budget, for a few per cent of throughput and p99.
DEFAULT_ACTIVE_NODES = 8 << 20


def choose_batch_variant(shapes):
    """Tile variant for a batch of (nx, ny) domains: the one with the least
    padded work, summed over the members' block tiles.  A tile's work is its
    marched rows (tile_y plus a halo row above and below each of its four
    warps) times its 32 lanes' columns, two columns per lane costing
    TWO_COLUMN_COST times four per column; the persistent batch kernel takes
    tiles from one work list, so the waves even out.  Between two variants
    of the same tiles, the one whose kernel also carries the clean-tile code
    wins: its clean tiles skip node types and wall terms, and the batch runs
    them after the others."""
    best, best_cost = 0, None
    for v in range(binding.lbm_variant_count()):
        tx, ty, cols = binding.lbm_variant_tile(v)
        tiles = sum(binding.lbm_tile_count(nx, ny, v) for nx, ny in shapes)
        cost = tiles * (ty + 8) * 32 * cols * (TWO_COLUMN_COST if cols == 2
                                               else 1.0)
        if best_cost is None or cost < best_cost or (
                cost == best_cost and binding.lbm_variant_has_clean_code(v)
                and not binding.lbm_variant_has_clean_code(best)):
            best, best_cost = v, cost
    return best


def _start(req, stream):
    prob = req.problem()
    dom = binding.Domain.from_problem(prob, stream=stream)
    return dom, prob


class Server:
    def __init__(self, capacity=256, max_tiles=1 << 20, chunk=200,
                 residual_tol=1e-7, max_steps=20000, hbm_budget=None,
                 keep_states=False, policy="sjf",
                 max_active_nodes=DEFAULT_ACTIVE_NODES, max_wait=2.0):
        import torch
        self.torch = torch
        self.stream = torch.cuda.Stream()
        self.batch = binding.Batch(capacity, max_tiles, stream=self.stream)
        self.capacity = capacity
        self.chunk = int(chunk)
        self.tol = float(residual_tol)
        self.max_steps = int(max_steps)
        # a fixed budget when given; else each admission asks the device
        # how much memory is free at that moment (free_bytes)
        self.budget = int(hbm_budget) if hbm_budget else None
        self.reserve = 1 << 30  # kept free for the rest of the process
        self.keep_states = keep_states
        self.policy = policy
        self.max_nodes = int(max_active_nodes) if max_active_nodes else None
        self.max_wait = float(max_wait)
        self.auto_variant = True

    def free_bytes(self):
        """Device memory a new request may take now: what the driver
        reports free plus what PyTorch's caching allocator holds unused,
        less a reserve."""
        torch = self.torch
        free, _ = torch.cuda.mem_get_info()
        cached = torch.cuda.memory_reserved() - torch.cuda.memory_allocated()
        return free + cached - self.reserve

    def run(self, requests, clock=time.perf_counter, on_done=None):
        """Serves `requests` (with arrival times in seconds from now);
        returns one Result per request, in request order.  `on_done`, if
        given, is called with each Result as its request completes."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = []
        active = {}  # slot -> [req, dom, steps, admitted, bytes]
        used = 0
        nodes = 0
        done = {}
        t0 = clock()
        changed = False
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting and len(active) < self.capacity:
                req = select_next(waiting, now, self.policy, self.max_wait)
                need = _footprint(req)
                size = req.nx * req.ny
                fits = (used + need <= self.budget if self.budget is not None
                        else need <= self.free_bytes())
                if active and (not fits or
                               (self.max_nodes is not None and
                                nodes + size > self.max_nodes)):
                    break  # wait for memory or node budget to free up
                waiting.remove(req)
                dom, _ = _start(req, self.stream)
                slot = self.batch.add(dom)
                active[slot] = [req, dom, 0, clock() - t0, need]
                used += need
                nodes += size
                changed = True
            if not active:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                continue
            if changed and self.auto_variant:
                self.batch.set_variant(choose_batch_variant(
                    [(e[0].nx, e[0].ny) for e in active.values()]))
            changed = False
            self.batch.step(self.chunk)
            res, _, status = self.batch.residuals()
            for slot in list(active):
                entry = active[slot]
                entry[2] += self.chunk
                req, dom, steps = entry[0], entry[1], entry[2]
                if status[slot] not in (binding.LBM_OK,):
                    raise binding.LbmError(int(status[slot]),
                                           "request %d" % req.rid)
                converged = res[slot] <= self.tol
                if converged or steps >= self.max_steps:
                    state = dom.get_state() if self.keep_states else None
                    if not self.keep_states:
                        dom.moments()  # the result goes back to the client
                    t = clock() - t0
                    done[req.rid] = Result(req.rid, req.arrival, entry[3], t,
                                           steps, float(res[slot]), converged,
                                           req.nx * req.ny, state)
                    if on_done is not None:
                        on_done(done[req.rid])
                    self.batch.remove(slot)
                    dom.close()
                    used -= entry[4]
                    nodes -= req.nx * req.ny
                    del active[slot]
                    changed = True
        return [done[r.rid] for r in requests]

    def close(self):
        self.batch.close()


def serve_sequential(requests, chunk=200, residual_tol=1e-7, max_steps=20000,
                     clock=time.perf_counter, keep_states=False, on_done=None):
    """The plain form: one request at a time, in arrival order."""
    import torch
    stream = torch.cuda.Stream()
    out = {}
    t0 = clock()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        admitted = clock() - t0
        dom, _ = _start(req, stream)
        steps, res = 0, float("inf")
        while True:
            dom.step(chunk)
            steps += chunk
            res, _ = dom.residual()
            if res <= residual_tol or steps >= max_steps:
                break
        state = dom.get_state() if keep_states else None
        if not keep_states:
            dom.moments()
        out[req.rid] = Result(req.rid, req.arrival, admitted, clock() - t0,
                              steps, float(res), res <= residual_tol,
                              req.nx * req.ny, state)
        if on_done is not None:
            on_done(out[req.rid])
        dom.close()
    return [out[r.rid] for r in requests]


def summary(results):
    lat = np.array([r.latency for r in results])
    makespan = max(r.completed for r in results)
    return {"requests": len(results),
            "solves_per_s": round(len(results) / makespan, 3),
            "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "makespan_s": round(makespan, 3),
            "converged": int(sum(r.converged for r in results)),
            "capped": int(sum(not r.converged for r in results)),
            "lattice_updates": int(sum(r.steps * r.nodes for r in results))}
