"""Continuous-batching service for LBMTau1 solves.

Requests (a domain to solve to a steady-state residual) arrive over time.
The service keeps every admitted domain's fields on the device and advances
all of them together with the batched step (one launch per time step for the
whole batch, lbm_batch_step).  Between chunks of steps it reads every member's
residual with one copy, retires the converged members (their final state is
downloaded and their memory freed), and admits waiting requests while batch
slots and the device-memory budget allow: new work joins while older work is
still on the device.  All arithmetic runs in the library's kernels; this
module only schedules.

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


def _start(req, stream):
    prob = req.problem()
    dom = binding.Domain.from_problem(prob, stream=stream)
    return dom, prob


class Server:
    def __init__(self, capacity=256, max_tiles=1 << 20, chunk=200,
                 residual_tol=1e-7, max_steps=20000, hbm_budget=None,
                 keep_states=False):
        import torch
        self.torch = torch
        self.stream = torch.cuda.Stream()
        self.batch = binding.Batch(capacity, max_tiles, stream=self.stream)
        self.capacity = capacity
        self.chunk = int(chunk)
        self.tol = float(residual_tol)
        self.max_steps = int(max_steps)
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(hbm_budget) if hbm_budget else int(0.8 * free)
        self.keep_states = keep_states

    def run(self, requests, clock=time.perf_counter):
        """Serves `requests` (with arrival times in seconds from now);
        returns one Result per request, in request order."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active = {}  # slot -> [req, dom, steps, admitted, bytes]
        used = 0
        done = {}
        t0 = clock()
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting and len(active) < self.capacity:
                need = _footprint(waiting[0])
                if used + need > self.budget and active:
                    break  # wait for memory to free up
                req = waiting.popleft()
                dom, _ = _start(req, self.stream)
                slot = self.batch.add(dom)
                active[slot] = [req, dom, 0, clock() - t0, need]
                used += need
            if not active:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                continue
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
                    self.batch.remove(slot)
                    dom.close()
                    used -= entry[4]
                    del active[slot]
        return [done[r.rid] for r in requests]

    def close(self):
        self.batch.close()


def serve_sequential(requests, chunk=200, residual_tol=1e-7, max_steps=20000,
                     clock=time.perf_counter, keep_states=False):
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
