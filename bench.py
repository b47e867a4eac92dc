"""Benchmark of the LBMTau1 D2Q9 step on GB300.

One bench step is one full LBMTau1 time step over the whole domain through the
C ABI (``lbm_step(ctx, 1)``): the fused pull / equilibrium / wall rule /
moment accumulation kernel with its fused residual and mass reduction, plus
the one-block FP64 finalize kernel.

Workload: the lid-driven cavity of Section 3 (walls on three sides, a fixed
lid row moving at u = 0.1), FP32 storage, at the largest size of the
256^2 .. 16384^2 single-domain sweep, 16384^2 nodes (6.7 GB of fields and node
types, far larger than the 129 MB L2, so no L2 flush is needed between steps).
Beside it: the single-domain bandwidth sweep (fully periodic boxes with a
small random perturbation, 256^2 .. 16384^2, FP32, FP16 and BF16 storage;
sizes that fit in L2 are marked as such and say nothing about HBM), the
1024^2 cavity over its 20000 steps, the storage precision on the Poiseuille
channel, the batched 512-domain configuration (FP32 and FP16) and the serving
loop.

Multi-GPU: the step does not shard here (one domain per GPU); ``--gpus N``
under torchrun runs N independent replicas (weak scaling) and reports the sum
of their throughputs over the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (per step, one oracle step over the top 256 rows of the cavity, full
width), so that the default 2000 steps end within a few minutes.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9 LBMTau1 MLUPS & % HBM roofline; batched solves/s, p99 vs plain"
UNIT = "MLUPS"
BYTES_PER_LUP = 24          # read + write rho-1, jx, jy (FP32)
MASK_BYTES_PER_LUP = 1      # the node type, read by tiles with walls only
FALLBACK_HBM_GBS = 6800.0   # used only when MEASURED_PEAKS.json is absent
KERNEL_SRC = os.path.join(ROOT, "paper_1912_09327_gb300", "csrc",
                          "lbm_kernels.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "lbm_step_kernel_f32.traffic.txt")


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=16384)
    ap.add_argument("--e2e-steps", type=int, default=24)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batched-domains", type=int, default=512)
    ap.add_argument("--batched-steps", type=int, default=2000)
    ap.add_argument("--porous-cap", type=int, default=50000,
                    help="step cap of the porous run to residual 1e-8")
    ap.add_argument("--serving-requests", type=int, default=32)
    ap.add_argument("--serving-cap", type=int, default=10000,
                    help="step cap per served request")
    ap.add_argument("--serving-full", action="store_true",
                    help="configuration 5 as stated: 256 requests, each run "
                         "to residual 1e-7 (cap 4e6 steps, far above what "
                         "any request needs); takes tens of minutes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int) -> float:
    """Slowest rank's time (the whole job ends when the last replica does)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def load_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
                if k in d:
                    return float(d[k]), "measured (MEASURED_PEAKS.json %s)" % k
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback (no MEASURED_PEAKS.json)"


def kernel_hash(path=KERNEL_SRC):
    """Hash of the kernel source's code (comment-only lines and blank lines
    left out, so that editing a comment does not invalidate a profile)."""
    code = [l.rstrip() for l in open(path).read().splitlines()
            if l.strip() and not l.strip().startswith("//")]
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def load_traffic(nodes):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    domain by its node count; None when the kernel changed since."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    for line in open(TRAFFIC_FILE):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256_16") != kernel_hash():
        return None
    try:
        return float(kv["dram_bytes_per_node"]) * nodes
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                    "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def time_steps(dom, stream, steps):
    """Per-step CUDA-event durations (ms) of lbm_step(ctx, 1) on the domain's
    stream."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        dom.step(1)
        b.record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def bytes_per_lup(storage="f32"):
    """Algorithmic bytes per lattice update: rho - 1, jx, jy read and written
    in the storage format (the paper's 2 N_f c per node, Eq. LBMTau1memory);
    the node type (1 B, read only by tiles with walls) is not counted."""
    return 6 * {"f32": 4, "f16": 2, "bf16": 2}[storage]


def problem_domain(binding, p, stream, storage="f32"):
    ny, nx = p.mask.shape
    d = binding.Domain(nx, ny, p.periodic, p.force, stream=stream,
                       storage=storage)
    d.set_geometry(p.mask)
    d.set_moments(p.rho, p.jx, p.jy)
    return d


def cavity_domain(binding, n, stream, storage="f32"):
    from paper_1912_09327_gb300 import workloads as wl
    p = wl.cavity(n, 0.1)
    return problem_domain(binding, p, stream, storage), p


def run_sweep(binding, stream, sizes, storage="f32", steps=200):
    """Single-domain bandwidth sweep: fully periodic all-fluid boxes with a
    small random perturbation (delta rho, u ~ 1e-3 N(0, 1)), n x n for each
    size, in one storage format; `steps` timed steps after 20 warm-up steps
    (the time of lbm_step(ctx, steps), one reduction at its end)."""
    from paper_1912_09327_gb300 import workloads as wl
    out = {}
    import torch
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    bpl = bytes_per_lup(storage)
    for n in sizes:
        d = problem_domain(binding, wl.periodic_box_tiled(n), stream, storage)
        d.step(20)
        stream.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        d.step(steps)
        e.record(stream)
        stream.synchronize()
        ms = s.elapsed_time(e)
        ws = bpl * n * n
        out[str(n)] = {"mlups": round(n * n * steps / (ms * 1e3), 1),
                       "gbs_algorithmic": round(ws / (ms / steps) / 1e6, 1),
                       "l2_resident": bool(2 * ws < l2),
                       "variant": d.variant()}
        d.close()
        del d
        torch.cuda.empty_cache()
    return {"workload": "fully periodic all-fluid n^2 box, random "
                        "perturbation 1e-3, %s storage, %d timed steps"
                        % (storage, steps),
            "bytes_per_lup": bpl, "sizes": out}


def run_cavity(binding, stream, n=1024, steps=20000):
    """The lid-driven cavity configuration itself: n x n, lid u = 0.1, FP32,
    all its steps in one lbm_step call (the working set fits in L2)."""
    import torch
    d, _ = cavity_domain(binding, n, stream)
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    s.record(stream)
    d.step(steps)
    e.record(stream)
    res, mass = d.residual()
    ms = s.elapsed_time(e)
    out = {"workload": "lid-driven cavity %dx%d, lid u=0.1, FP32, %d steps "
                       "(one lbm_step call)" % (n, n, steps),
           "seconds": round(ms / 1e3, 4),
           "mlups": round(n * n * steps / (ms * 1e3), 1),
           "residual_last_step": res, "variant": d.variant()}
    d.close()
    return out


def run_precision(binding, stream, max_steps=60000, chunk=5000):
    """Storage precision on the Poiseuille channel 64 x 32 (u_max 0.01): run
    to steady state (residual <= 1e-12, or max_steps) in each storage format
    (16-bit: stochastic rounding, the default, and round-to-nearest),
    then the relative velocity error against the exact discrete steady state
    of the method, U(y) = 3 f y (H - y) - f with rho = 1 (it holds for the
    wall rule of Eq. feqnoslip, so the FP32 figure is rounding alone), and
    against the plane-Poiseuille parabola u = 3 f y (H - y) (nu = 1/6), whose
    gap to the former is the method's own 4 / (3 H^2) discretisation error."""
    from paper_1912_09327_gb300 import workloads as wl
    p = wl.channel(64, 32, 0.01)
    f = p.force[0]
    H = p.meta["H"]
    y = np.arange(1, H)
    parabola = 3.0 * f * y * (H - y)
    exact = parabola - f
    out = {"workload": "Poiseuille channel 64x32 (x-periodic, walls at "
                       "y = 0 and 31), u_max 0.01, run to residual 1e-12"}
    for storage, rounding in (("f32", "nearest"), ("f16", "stochastic"),
                              ("bf16", "stochastic"), ("f16", "nearest"),
                              ("bf16", "nearest")):
        ny_, nx_ = p.mask.shape
        d = binding.Domain(nx_, ny_, p.periodic, p.force, stream=stream,
                           storage=storage, rounding=rounding)
        d.set_geometry(p.mask)
        d.set_moments(p.rho, p.jx, p.jy)
        steps, res = 0, float("inf")
        while steps < max_steps:
            d.step(chunk)
            steps += chunk
            res, _ = d.residual()
            if res <= 1e-12:
                break
        R, U, _ = d.moments()
        d.close()
        u = (U / R)[1:H, :]
        key = storage if rounding == "stochastic" or storage == "f32" \
            else storage + "_nearest"
        out[key] = {
            "rounding": rounding if storage != "f32" else "fp32",
            "steps": steps, "residual": res,
            "err_vs_exact_steady_state": float(
                np.abs(u - exact[:, None]).max() / exact.max()),
            "err_vs_parabola": float(
                np.abs(u - parabola[:, None]).max() / parabola.max())}
    out["method_discretisation_error"] = 4.0 / (3.0 * H * H)
    return out


def run_e2e(binding, dom, n, steps, lanes=2):
    """Same metric through the public API with host buffers: per step, the
    exact state goes host -> device from pinned memory (lbm_set_state), one
    lbm_step, the state comes back (lbm_get_state) and the residual is read
    (lbm_residual); wall-clock time with the copies inside.  `lanes`
    independent cavity domains are in flight, each driven by its own host
    thread (the library's calls release the interpreter lock and block only
    the calling thread), so that one domain's upload overlaps another's
    download on the host link; `steps` steps in all, split between them."""
    import threading
    import torch
    doms = [dom] + [cavity_domain(binding, n, torch.cuda.Stream())[0]
                    for _ in range(lanes - 1)]
    per = max(1, -(-steps // lanes))
    bufs = []
    for d in doms:
        bi = [torch.empty((n, n), dtype=torch.float32, pin_memory=True)
              for _ in range(3)]
        bo = [torch.empty((n, n), dtype=torch.float32, pin_memory=True)
              for _ in range(3)]
        binding.lbm_get_state(d.ctx, *bi)
        binding.lbm_set_state(d.ctx, *bi)
        d.step(1)
        d.residual()
        bufs.append((bi, bo))
    torch.cuda.synchronize()
    errors = []
    start = threading.Barrier(lanes + 1)

    def lane(d, bi, bo):
        try:
            start.wait()
            for _ in range(per):
                binding.lbm_set_state(d.ctx, *bi)
                d.step(1)
                binding.lbm_get_state(d.ctx, *bo)
                d.residual()
        except Exception as e:  # reported after the join
            errors.append(e)

    threads = [threading.Thread(target=lane, args=(d, bi, bo))
               for d, (bi, bo) in zip(doms, bufs)]
    for t in threads:
        t.start()
    start.wait()
    t0 = time.perf_counter()
    for t in threads:
        t.join()
    dt = time.perf_counter() - t0
    for d in doms[1:]:
        d.close()
    if errors:
        raise errors[0]
    total = per * lanes
    h2d = 3 * 4 * n * n
    d2h = 3 * 4 * n * n + 32
    return {"value": round(n * n * total / dt / 1e6, 1), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": total, "domains_in_flight": lanes,
            "api": "lbm_set_state + lbm_step(1) + lbm_get_state + lbm_residual, "
                   "pinned host, one host thread per domain"}


def run_multiphase(binding, stream, n=4096, steps=200):
    """The multiphase drop of Section 4 (liquid disc in its periodic vapour,
    Shan-Chen coupling g = -5), n x n, FP32: MLUPS of lbm_step(ctx, steps)
    (one reduction at the end) beside the single-phase step on a periodic
    box of the same size, after 200 steps that form the interface."""
    import torch
    from paper_1912_09327_gb300 import workloads as wl
    out = {"workload": "drop in periodic vapour %dx%d, g = -5, FP32, %d timed "
                       "steps (one reduction at the end)" % (n, n, steps)}
    for name, p in (("multiphase", wl.drop(n)),
                    ("single_phase", wl.periodic_box_tiled(n))):
        d = binding.Domain.from_problem(p, stream=stream)
        d.step(200)
        stream.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        d.step(steps)
        e.record(stream)
        stream.synchronize()
        ms = s.elapsed_time(e)
        res, mass = d.residual()
        out[name] = {"mlups": round(n * n * steps / (ms * 1e3), 1),
                     "ms_per_step": round(ms / steps, 4),
                     "variant": d.variant(), "residual": res}
        d.close()
        torch.cuda.empty_cache()
    out["multiphase_over_single"] = round(out["multiphase"]["mlups"] /
                                          out["single_phase"]["mlups"], 3)
    return out


def run_porous(binding, stream, n=4096, tol=1e-8, cap=50000, check=2000):
    """The porous-medium configuration: n x n periodic sample of seeded discs
    (radius 8..24, solid fraction 0.30), force 1e-5, run in FP32 to residual
    `tol` (checked every `check` steps, capped at `cap`), with the Reynolds
    number <u_x> D / nu of the result; then FP16 and BF16 storage (stochastic
    rounding) for the same number of steps, their velocity error reported
    against the FP32 field (which matches the FP64 oracle to FP32 rounding,
    tests).  16-bit storage cannot meet a 1e-8 residual (its rounding noise is
    about one unit in the last place per step)."""
    import torch
    from paper_1912_09327_gb300 import workloads as wl
    p = wl.porous(n, seed=0)
    fluid = p.mask == wl.FLUID
    out = {"workload": "porous %dx%d, %d discs, solid fraction %.3f, mean "
                       "diameter %.1f, force 1e-5, residual %.0e (cap %d)"
                       % (n, n, p.meta["discs"], p.meta["solid_fraction"],
                          p.meta["mean_diameter"], tol, cap)}
    ref = None
    steps_done = None
    for storage in ("f32", "f16", "bf16"):
        d = problem_domain(binding, p, stream, storage)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        s.record(stream)
        steps, res = 0, float("inf")
        target = steps_done if steps_done else cap
        while steps < target:
            d.step(check)
            steps += check
            res, _ = d.residual()
            if storage == "f32" and res <= tol:
                break
        e.record(stream)
        stream.synchronize()
        sec = s.elapsed_time(e) / 1e3
        R, U, V = d.moments()
        d.close()
        ux = U / R
        entry = {"steps": steps, "residual": res, "seconds": round(sec, 3),
                 "mlups": round(n * n * steps / sec / 1e6, 1)}
        if storage == "f32":
            steps_done = steps
            ref = ux
            entry["converged"] = bool(res <= tol)
            entry["mean_ux_fluid"] = float(ux[fluid].mean())
            entry["reynolds"] = float(ux[fluid].mean() * p.meta["mean_diameter"]
                                      * 6.0)
        else:
            dif = np.abs(ux - ref)[fluid]
            scale = np.abs(ref[fluid]).max()
            entry["err_vs_f32_max"] = float(dif.max() / scale)
            entry["err_vs_f32_mean"] = float(dif.mean() / np.abs(ref[fluid]).mean())
        out[storage] = entry
        torch.cuda.empty_cache()
    return out


def run_batched(binding, domains, steps, storage="f32"):
    """Configuration: 512 independent domains (seeded thirds of channels,
    cavities and porous samples, sides log-uniform in [64, 1024]), 2000 steps
    each, in one storage format; batched (one launch per step for all
    domains, autotuned tile variant) against the plain form (one domain after
    another, lbm_step)."""
    import torch
    from paper_1912_09327_gb300 import workloads as wl
    probs = wl.batch_mix(domains, seed=0)
    nodes = sum(p.mask.size for p in probs)
    stream = torch.cuda.Stream()
    doms = [binding.Domain.from_problem(p, stream=stream, storage=storage)
            for p in probs]
    tiles = sum(binding.lbm_tile_count(p.mask.shape[1], p.mask.shape[0])
                for p in probs)   # the most over the variants the autotuner tries
    batch = binding.Batch(len(doms), tiles, stream=stream)
    for d in doms:
        batch.add(d)
    chosen, tuned = batch.autotune(10)
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(steps)
    e1.record(stream)
    batch.residuals()  # syncs; every member's residual of the last step
    t_batch = e0.elapsed_time(e1) / 1e3
    batch.close()
    for d in doms:
        d.close()
    torch.cuda.empty_cache()
    # the plain form, one domain after another, every one of its steps timed
    doms = [binding.Domain.from_problem(p, stream=stream, storage=storage)
            for p in probs]
    stream.synchronize()
    e0.record(stream)
    for d in doms:
        d.step(steps)
    e1.record(stream)
    stream.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    for d in doms:
        d.close()
    torch.cuda.empty_cache()
    return {"workload": "%d domains (channel/cavity/porous thirds, sides "
                        "log-uniform 64..1024), %d steps each, %s storage"
                        % (domains, steps, storage),
            "nodes": int(nodes), "variant": chosen,
            "autotune_ms_per_step": [round(t, 4) for t in tuned],
            "batched_s": round(t_batch, 4), "plain_s": round(t_plain, 4),
            "plain_timed_steps": steps,
            "solves_per_s_batched": round(domains / t_batch, 2),
            "solves_per_s_plain": round(domains / t_plain, 2),
            "mlups_batched": round(nodes * steps / t_batch / 1e6, 1),
            "mlups_plain": round(nodes * steps / t_plain / 1e6, 1),
            "speedup": round(t_plain / t_batch, 2)}


def run_serving(requests_n, cap=10000, full=False):
    """Configuration: Poisson arrivals (seeded, 200 requests/s) of channel,
    cavity and porous solves with sides log-uniform in [64, 2048], each run to
    residual 1e-7 (capped at `cap` steps, reported), admitted by free device
    memory; continuous batching against the plain sequential form.  `full`:
    the processor-sharing comparison is left out (its time is the same)."""
    from paper_1912_09327_gb300 import serving, workloads as wl
    reqs = wl.request_stream(requests_n, rate=200.0, seed=0)
    kinds = {q.rid: q for q in reqs}

    def log(form):
        def on_done(r):   # progress on stderr: long runs leave a record
            q = kinds[r.rid]
            print("serving %s: request %d %s %dx%d done after %d steps, "
                  "residual %.3g, latency %.3f s" % (form, r.rid, q.kind, q.nx,
                                                    q.ny, r.steps, r.residual,
                                                    r.latency),
                  file=sys.stderr, flush=True)
        return on_done if full else None

    srv = serving.Server(capacity=max(requests_n, 8), chunk=200,
                         residual_tol=1e-7, max_steps=cap)
    batched_results = srv.run(reqs, on_done=log("batched"))
    batched = serving.summary(batched_results)
    srv.close()
    shared = None
    if not full:
        # every request admitted at once, in arrival order (processor sharing)
        srv = serving.Server(capacity=max(requests_n, 8), chunk=200,
                             residual_tol=1e-7, max_steps=cap, policy="fifo",
                             max_active_nodes=None)
        shared = serving.summary(srv.run(reqs))
        srv.close()
    plain = serving.summary(serving.serve_sequential(reqs, chunk=200,
                                                     residual_tol=1e-7,
                                                     max_steps=cap,
                                                     on_done=log("plain")))
    return {"workload": "%d requests, Poisson 200/s, sides log-uniform "
                        "64..2048, residual 1e-7, cap %d steps, chunk 200"
                        % (requests_n, cap),
            "continuous_batching": batched,
            "policy": "smallest first, %d Mi active nodes, 2 s wait bound"
                      % (serving.DEFAULT_ACTIVE_NODES >> 20),
            "continuous_batching_fifo_unbounded": shared,
            "plain_sequential": plain,
            "per_request": [{"rid": r.rid, "kind": q.kind, "nx": q.nx,
                             "ny": q.ny, "steps": r.steps,
                             "residual": r.residual,
                             "latency_s": round(r.latency, 4)}
                            for q, r in zip(reqs, batched_results)]
            if full else None}


def cpu_baseline(size, rows=1024, seconds=10.0):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample:
    whole steps over the top `rows` rows of the size x size cavity (full
    width), repeated until about `seconds` of CPU time have passed."""
    import oracle
    from paper_1912_09327_gb300 import workloads as wl
    p = wl.cavity(size, 0.1, ny=rows)
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    R, U, V = p.state()
    oracle.run(p.mask, R, U, V, 1, p.periodic, p.force)   # warm-up
    steps = 0
    t0 = time.perf_counter()
    while steps < 2 or time.perf_counter() - t0 < seconds:
        R, U, V = oracle.run(p.mask, R, U, V, 1, p.periodic, p.force)
        steps += 1
    dt = time.perf_counter() - t0
    cores_used = oracle.max_threads()
    # the same oracle on one core, over a quarter of the time
    oracle.set_threads(1)
    R, U, V = p.state()
    steps1 = 0
    t0 = time.perf_counter()
    while steps1 < 1 or time.perf_counter() - t0 < seconds / 4:
        R, U, V = oracle.run(p.mask, R, U, V, 1, p.periodic, p.force)
        steps1 += 1
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return {"value": round(size * rows * steps / dt / 1e6, 2), "unit": UNIT,
            "cores": cores_used, "kind": "oracle",
            "value_1_core": round(size * rows * steps1 / dt1 / 1e6, 2),
            "sample": "%d steps (%d on one core) of the top %d rows (full "
                      "width %d) of the lid-driven cavity, FP64 C oracle, "
                      "OpenMP over rows" % (steps, steps1, rows, size)}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1912_09327_gb300 import workloads as wl
    import oracle
    oracle.build()
    size, rows = args.size, 256
    p = wl.cavity(size, 0.1, ny=rows)
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    R, U, V = p.state()
    for _ in range(max(args.warmup, 0)):
        R, U, V = oracle.run(p.mask, R, U, V, 1, p.periodic, p.force)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        R, U, V = oracle.run(p.mask, R, U, V, 1, p.periodic, p.force)
    dt = time.perf_counter() - t0
    value = size * rows * args.steps / dt / 1e6
    sample = ("each step: one FP64 oracle step over the top %d rows (full "
              "width %d) of the %d^2 lid-driven cavity" % (rows, size, size))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 2),
            "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(size),
            "cpu_baseline": {"value": round(value, 2), "unit": UNIT,
                             "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 2), "unit": UNIT,
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(size):
    return {"workload": "D2Q9 LBMTau1 lid-driven cavity, lid u=0.1, FP32 "
                        "storage, %dx%d nodes (largest point of the "
                        "256^2-16384^2 single-domain sweep of the 1024^2 "
                        "cavity configuration)" % (size, size),
            "nx": size, "ny": size, "lid_u": 0.1, "storage": "f32",
            "l2": "inputs larger than L2 (%.1f GB working set vs 129 MB L2)"
                  % (BYTES_PER_LUP * size * size / 1e9),
            "parallelism": "replicas"}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return rc

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09327_gb300 import binding
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    n = args.size
    dom, _ = cavity_domain(binding, n, stream)

    for _ in range(max(args.warmup, 3)):
        dom.step(1)
    stream.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        per_step = time_steps(dom, stream, args.steps)
        t1.record(stream)
        stream.synchronize()
    total_ms = t0.elapsed_time(t1)
    torch.cuda.synchronize()
    barrier(world)
    total_ms = max_over_ranks(total_ms, world)
    res, mass = dom.residual()
    clocks = clk.summary()
    # the step kernel alone, without the per-step reduction: lbm_step(ctx, K)
    # reduces only on its last step
    ku = 100
    u0 = torch.cuda.Event(enable_timing=True)
    u1 = torch.cuda.Event(enable_timing=True)
    u0.record(stream)
    dom.step(ku)
    u1.record(stream)
    stream.synchronize()
    unreduced_ms = u0.elapsed_time(u1) / ku

    nodes = n * n
    value = nodes * args.steps * world / (total_ms * 1e3)
    kernel_ms = statistics.mean(per_step)
    peak, peak_src = load_peak()
    achieved = BYTES_PER_LUP * nodes / (kernel_ms * 1e-3) / 1e9
    traffic = load_traffic(nodes)
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": workload_config(n),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": traffic,
                         "kernel": "lbm_step_kernel<reduce> + finalize "
                                   "(events around lbm_step(ctx, 1))",
                         "algorithmic_bytes_per_launch": BYTES_PER_LUP * nodes,
                         "peak_source": peak_src},
            "unreduced_step": {
                "ms": round(unreduced_ms, 4),
                "mlups": round(n * n / (unreduced_ms * 1e3), 1),
                "gbs_algorithmic": round(BYTES_PER_LUP * n * n / (unreduced_ms * 1e-3) / 1e9, 1),
                "note": "lbm_step(ctx, 100) / 100: the step kernel without the residual reduction (it runs on the last step only)"},
            "step_variant": dom.variant(),
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
            "residual_last_step": res}

    if rank == 0:
        line["e2e"] = run_e2e(binding, dom, n, args.e2e_steps)
    dom.close()
    del dom
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_sweep:
        sizes = [256, 512, 1024, 2048, 4096, 8192, 16384]
        line["sweep"] = run_sweep(binding, stream, sizes)
        line["sweep_f16"] = run_sweep(binding, stream, sizes, "f16")
        line["sweep_bf16"] = run_sweep(binding, stream, sizes, "bf16")
        line["cavity_1024"] = run_cavity(binding, stream)
        line["porous_4096"] = run_porous(binding, stream, cap=args.porous_cap)
        line["multiphase_4096"] = run_multiphase(binding, stream)
        line["precision"] = run_precision(binding, stream)
    if rank == 0 and not args.no_batched:
        line["batched"] = run_batched(binding, args.batched_domains,
                                      args.batched_steps)
        line["batched_f16"] = run_batched(
            binding, args.batched_domains, args.batched_steps, storage="f16")
    if rank == 0 and not args.no_serving:
        if args.serving_full:
            line["serving"] = run_serving(256, cap=4000000, full=True)
        else:
            line["serving"] = run_serving(args.serving_requests,
                                          cap=args.serving_cap)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
