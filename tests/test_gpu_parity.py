"""Parity of the sm_103a LBMTau1 kernels (through the C ABI) with the FP64
CPU oracle, element by element on the same seeded inputs.

Tolerances.  The device stores rho - 1 and j in FP32 and computes in FP32.
- The channel case uses the bound the method is held to:
  max|u_gpu - u_oracle| / max|u_oracle| <= 1e-5 after the full run.
- General cases compare rho, jx, jy absolutely.  With field amplitude a (rho
  - 1 and j of order a), one FP32 step evaluates each output as about 30
  rounded operations on terms of size <= 6a (3 |j_P - j_O| and the like), so a
  forward bound is 30 * 2^-24 * 6a = 1.1e-5 a per step; independent roundings
  accumulate like a random walk over n steps.  The tests allow
  2e-6 * a * sqrt(n) + 1e-9, a fifth of the forward bound (observed: at most
  6.3e-7 a for one step on random fields).  The initial state's rounding to
  FP32 (3e-8 a) is inside this.
"""
import numpy as np
import pytest

import oracle
from paper_1912_09327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09327_gb300 import binding as b
    return b


def tolerance(amp, nsteps):
    return 2e-6 * amp * np.sqrt(nsteps) + 1e-9


def run_gpu(binding, prob, nsteps):
    d = binding.Domain.from_problem(prob)
    d.step(nsteps)
    out = d.moments()
    res = d.residual() if nsteps > 0 else None
    d.close()
    return out, res


def velocity_error(a, b):
    ua = np.stack([a[1] / a[0], a[2] / a[0]])
    ub = np.stack([b[1] / b[0], b[2] / b[0]])
    return np.abs(ua - ub).max() / np.abs(ub).max()


@pytest.mark.parametrize("rounding", ["nearest", "stochastic"])
def test_channel_64x32_5000_steps(binding, rounding):
    """Poiseuille channel, 64 x 32, 5000 steps, u_max ~ 0.01, FP32 storage
    rounded to nearest (the default) and stochastically."""
    p = wl.channel(64, 32, 0.01)
    d = binding.Domain.from_problem(p, rounding=rounding)
    d.step(5000)
    g = d.moments()
    res, mass = d.residual()
    d.close()
    o = oracle.run(p.mask, *p.state(), 5000, p.periodic, p.force)
    err = velocity_error(g, o)
    assert err <= 1e-5, err
    fluid = p.mask == 0
    # sum of FP32 rho - 1 over 5000 steps: within the FP32 unit roundoff
    assert mass == pytest.approx(o[0][fluid].sum(), rel=1e-7)


SIZES = [(1, 1), (2, 3), (3, 5), (4, 4), (17, 13), (121, 37), (119, 129),
         (250, 131), (241, 300), (480, 129)]


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("periodic", [(True, True), (False, False),
                                      (True, False), (False, True)])
def test_random_domains(binding, nx, ny, periodic):
    """Random node types (solid 20 %, fixed 5 %), random state, force, every
    periodicity, sizes spanning several 120 x 128 tiles and ragged tails."""
    amp, n = 0.02, 20
    p = wl.random_problem(nx, ny, seed=nx * 1000 + ny, amp=amp,
                          periodic=periodic, force=(1e-4, -5e-5))
    g, _ = run_gpu(binding, p, n)
    o = oracle.run(p.mask, *p.state(), n, p.periodic, p.force)
    tol = tolerance(amp, n)
    for a, b in zip(g, o):
        assert np.abs(a - b).max() <= tol


@pytest.mark.parametrize("nx,ny,periodic", [(301, 143, (True, False)),
                                             (1024, 1024, (False, False)),
                                             (37, 519, (True, True))])
def test_tile_variants_bit_identical(binding, nx, ny, periodic):
    """Every tile variant of the single-domain path gives the same state, bit
    for bit (each output node is computed by the same arithmetic, whatever
    tile holds it), and the automatic choice is one of them.  The residual
    and mass are sums whose grouping depends on the tile: each lane adds its
    own outputs in FP32 (at most 64 rows x 4 columns, a relative error below
    256 * 2^-24 = 1.5e-5 for the positive sums), the rest is FP64."""
    p = wl.random_problem(nx, ny, seed=nx + 7 * ny, amp=0.02,
                          periodic=periodic, force=(1e-4, -5e-5))
    nv = binding.lbm_variant_count()
    states, residuals = [], []
    for v in list(range(nv)) + [-1]:
        d = binding.Domain.from_problem(p)
        d.set_variant(v)
        chosen = d.variant()
        assert 0 <= chosen < nv and (v < 0 or chosen == v)
        d.step(9)
        states.append(d.get_state())
        residuals.append(d.residual())
        d.close()
    for st, r in zip(states[1:], residuals[1:]):
        for a, b in zip(st, states[0]):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        assert r[0] == pytest.approx(residuals[0][0], rel=1.5e-5)
        # mass: a signed sum of |rho - 1| <= 0.05 terms
        assert abs(r[1] - residuals[0][1]) <= 1.5e-5 * 0.05 * nx * ny
    o = oracle.run(p.mask, *p.state(), 9, p.periodic, p.force)
    g = [states[0][0].astype(np.float64) + 1.0,
         states[0][1].astype(np.float64), states[0][2].astype(np.float64)]
    solid = p.mask == wl.SOLID
    for a, b in zip(g, o):
        a[solid] = b[solid]   # solid nodes are stored as (0, -F), reported at rest
        assert np.abs(a - b).max() <= tolerance(0.02, 9)


NARROW = [1, 2, 3, 5, 7, 9, 15, 16, 17, 31, 33, 59, 61, 63, 65, 119, 121,
          123, 125, 127, 129, 241]


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_domain_edges_every_variant(binding, storage):
    """Widths around every tile and 16-byte boundary, periodic and walled in
    x: the clipped row windows and the wrapped columns -1 and nx give every
    tile variant the same state bit for bit, and (FP32) the oracle's."""
    nv = binding.lbm_variant_count()
    for i, nx in enumerate(NARROW):
        per = (i % 2 == 0, i % 3 == 0)
        p = wl.random_problem(nx, 23, seed=100 + nx, amp=0.02, periodic=per,
                              force=(1e-4, -5e-5))
        states = []
        for v in range(nv):
            d = binding.Domain(nx, 23, p.periodic, p.force, storage=storage)
            d.set_geometry(p.mask)
            d.set_moments(p.rho, p.jx, p.jy)
            d.set_variant(v)
            d.step(6)
            states.append(d.get_state())
            if v == 0 and storage == "f32":
                g = d.moments()
                o = oracle.run(p.mask, *p.state(), 6, p.periodic, p.force)
                for a, b in zip(g, o):
                    assert np.abs(a - b).max() <= tolerance(0.02, 6), (nx, per)
            d.close()
        for st in states[1:]:
            for a, b in zip(st, states[0]):
                assert np.array_equal(a.view(np.uint16 if a.itemsize == 2
                                             else np.uint32),
                                      b.view(np.uint16 if b.itemsize == 2
                                             else np.uint32)), (nx, per)


def test_clean_tile_kernel_on_large_domains(binding):
    """A domain large enough (here 8192^2: 2208 block tiles of the tall
    variant) whose warp tiles are mostly clean (interior, fluid only) gets
    the variant whose kernel also carries the code for clean tiles; it gives
    the state and the mass sum of the general kernel on the same tiles, bit
    for bit.  Its residual sums add the same non-negative terms in the same
    order in packed form, which the compiler may fuse with the scaling (one
    rounding instead of two), so the residual agrees to float rounding."""
    nx, ny = 8192, 8192
    p = wl.random_problem(nx, ny, seed=77, amp=0.02, p_solid=0.0, p_fixed=0.0,
                          periodic=(True, True), force=(1e-4, -5e-5))
    p.mask[1000:1010, 3000:3050] = wl.SOLID   # a few tiles with walls
    p.mask[4000, 100:140] = wl.FIXED
    d = binding.Domain.from_problem(p)
    v = d.variant()
    tx, ty, cols = binding.lbm_variant_tile(v)
    assert v != 0 and (tx, ty) == binding.lbm_variant_tile(0)[:2]
    d.step(6)
    got = d.get_state(), d.residual()
    d.close()
    d = binding.Domain.from_problem(p)
    d.set_variant(0)
    d.step(6)
    want = d.get_state(), d.residual()
    d.close()
    for a, b in zip(got[0], want[0]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert got[1][1] == want[1][1]
    assert got[1][0] == pytest.approx(want[1][0], rel=1e-6)


def test_graph_chunks_equal_direct_launches(binding):
    """On a capturable stream lbm_step replays runs of 16 inner steps from a
    captured CUDA graph; on the default stream it launches every step.  Both
    give the same state and residual bit for bit, also across calls of odd
    lengths (graphs for both starting copies) and a change of tile variant
    (the graphs are captured again)."""
    import torch
    p = wl.random_problem(333, 170, seed=41, amp=0.02, periodic=(True, False))
    runs = []
    for stream in (None, torch.cuda.Stream()):
        d = binding.Domain.from_problem(p, stream=stream)
        d.step(37)
        d.step(50)
        d.set_variant(2)
        d.step(40)
        runs.append((d.get_state(), d.residual()))
        d.close()
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert runs[0][1] == runs[1][1]


def test_single_step_exact_paths(binding):
    """One step on an all-fluid periodic box and on a walled box: every node
    is compared with the oracle."""
    for per in [(True, True), (False, False)]:
        p = wl.random_problem(300, 200, seed=5, p_solid=0.0, p_fixed=0.0,
                              amp=0.05, periodic=per, force=(0.0, 0.0))
        g, _ = run_gpu(binding, p, 1)
        o = oracle.step(p.mask, *p.state(), p.periodic, p.force)
        for a, b in zip(g, o):
            assert np.abs(a - b).max() <= tolerance(0.05, 1)


def sample_nodes(shape, count, seed=0):
    rng = np.random.default_rng(seed)
    return rng.choice(shape[0] * shape[1], size=count, replace=False)


def test_cavity_1024_full_size(binding):
    """Lid-driven cavity 1024^2, lid u = 0.1 (Section 3's cavity, Re = 614):
    every node against the oracle after the configuration's full 20000 steps,
    at the bound the method is held to, max|u_gpu - u_oracle| / max|u_oracle|
    <= 1e-5; on the way, the residual of every 2000-step call shrinks."""
    oracle.set_threads(oracle.max_threads())
    p = wl.cavity(1024, 0.1)
    d = binding.Domain.from_problem(p)
    res_prev = None
    for _ in range(10):
        d.step(2000)
        res, _ = d.residual()
        assert np.isfinite(res)
        if res_prev is not None:
            assert res < res_prev
        res_prev = res
    g = d.moments()
    d.close()
    o = oracle.run(p.mask, *p.state(), 20000, p.periodic, p.force)
    print("cavity 1024^2 x 20000 f32 max|du|/max|u| = %.3g"
          % velocity_error(g, o))
    assert velocity_error(g, o) <= 1e-5
    assert np.abs(g[0] - o[0]).max() <= 1e-5
    # 16-bit storage (stochastic rounding) against the same oracle state
    for fmt, bound in (("f16", 4e-3), ("bf16", 4e-2)):
        d = binding.Domain.from_problem(p, storage=fmt)
        d.step(20000)
        err = velocity_error(d.moments(), o)
        d.close()
        print("cavity 1024^2 x 20000", fmt, "max|du|/max|u| = %.3g" % err)
        assert err <= bound, (fmt, err)


def test_porous_4096_full_size(binding):
    """Periodic porous medium 4096^2 (seeded discs, solid fraction 0.30,
    f_x = 1e-5): every node against the oracle after 2000 steps at the
    1e-5 velocity bound; then on to 50000 steps (near the FP32 residual floor
    of this flow), where one more step is checked on 20000 sampled nodes
    against the oracle's single-node update, and the Reynolds number of the
    flow stays below 1."""
    oracle.set_threads(oracle.max_threads())
    p = wl.porous(4096, seed=0)
    d = binding.Domain.from_problem(p)
    d.step(2000)
    g = d.moments()
    o = oracle.run(p.mask, *p.state(), 2000, p.periodic, p.force)
    print("porous 4096^2 x 2000 f32 max|du|/max|u| = %.3g"
          % velocity_error(g, o))
    assert velocity_error(g, o) <= 1e-5
    assert np.abs(g[0] - o[0]).max() <= 1e-6
    for fmt, bound in (("f16", 4e-3), ("bf16", 4e-2)):
        d16 = binding.Domain.from_problem(p, storage=fmt)
        d16.step(2000)
        err = velocity_error(d16.moments(), o)
        d16.close()
        print("porous 4096^2 x 2000", fmt, "max|du|/max|u| = %.3g" % err)
        assert err <= bound, (fmt, err)
    del g, o
    d.step(47999)
    before = d.moments()
    d.step(1)
    after = d.moments()
    nodes = sample_nodes(p.mask.shape, 20000, seed=1)
    ref = oracle.step_nodes(p.mask, *before, nodes, p.periodic, p.force)
    for f in range(3):
        assert np.abs(after[f].ravel()[nodes] - ref[:, f]).max() <= 1e-9
    fluid = p.mask == 0
    u_mean = (after[1][fluid] / after[0][fluid]).mean()
    Re = u_mean * p.meta["mean_diameter"] / wl.NU
    assert 0 < Re < 1
    d.close()


def test_largest_sweep_domain_sampled(binding):
    """16384^2 all-fluid periodic box (the largest bandwidth-sweep domain):
    one step from a random state, 50000 sampled nodes against the oracle."""
    n = 16384
    rng = np.random.default_rng(7)
    amp = 1e-3
    st = [(amp * rng.standard_normal((n, n), dtype=np.float32))
          for _ in range(3)]
    mask = np.zeros((n, n), np.uint8)
    d = binding.Domain(n, n, (True, True), (0.0, 0.0))
    d.set_geometry(mask)
    d.set_state(*st)
    d.step(1)
    nodes = sample_nodes((n, n), 50000, seed=2)
    R0 = 1.0 + st[0].astype(np.float64)
    ref = oracle.step_nodes(mask, R0, st[1].astype(np.float64),
                            st[2].astype(np.float64), nodes, (True, True))
    del R0
    got = d.get_state()
    d.close()
    assert np.abs(got[0].ravel()[nodes].astype(np.float64) + 1.0
                  - ref[:, 0]).max() <= 1e-9
    assert np.abs(got[1].ravel()[nodes] - ref[:, 1]).max() <= 1e-9
    assert np.abs(got[2].ravel()[nodes] - ref[:, 2]).max() <= 1e-9


def test_periodic_invariants_gpu(binding):
    """All-fluid periodic box: mass conserved, total momentum grows by N*f
    per step (to FP32 roundoff)."""
    p = wl.periodic_box(257, 190, seed=4, amp=1e-2)
    force = (2e-5, -1e-5)
    d = binding.Domain(257, 190, (True, True), force)
    d.set_geometry(p.mask)
    d.set_moments(*p.state())
    m0 = p.rho.sum()
    jx0, jy0 = p.jx.sum(), p.jy.sum()
    n = 100
    d.step(n)
    _, mass = d.residual()
    R, U, V = d.moments()
    N = p.mask.size
    assert abs(mass - m0) / m0 < 1e-7
    assert abs(R.sum() - m0) / m0 < 1e-7
    assert abs(U.sum() - jx0 - n * N * force[0]) < 1e-7 * N * 1e-2
    assert abs(V.sum() - jy0 - n * N * force[1]) < 1e-7 * N * 1e-2
    d.close()


def test_order_one_density_deviations_keep_their_mass(binding):
    """A periodic box at density 0.5 +- 0.05 (a deviation rho - 1 of order
    one, as in a multiphase vapour; here single phase): after 3000 steps the
    stored mass is the initial one to 1e-6 (measured 6e-8: the rounding of
    deviations near -0.5, whose half ulp is 3e-8), and the reduced mass is
    the sum of the stored densities to 1e-8.  The density a node receives is
    the weighted sum of its sources'; with FP32 weights summing to
    1 + 7.5e-9 every step would scale the mean deviation -0.5 and the mass
    would drift by about 2e-5 here."""
    n = 192
    y, x = np.mgrid[0:n, 0:n]
    rho = 0.5 + 0.05 * np.sin(2 * np.pi * x / n) * np.cos(2 * np.pi * y / n)
    z = np.zeros_like(rho)
    mask = np.zeros((n, n), np.uint8)
    d = binding.Domain(n, n, (True, True), (0.0, 0.0))
    d.set_geometry(mask)
    d.set_moments(rho, z, z)
    m0 = d.moments()[0].sum()
    d.step(3000)
    _, mass = d.residual()
    m1 = d.moments()[0].sum()
    d.close()
    assert abs(m1 - m0) <= 1e-6 * m0
    assert abs(mass - m1) <= 1e-8 * m0


def test_quiescent_is_bit_exact(binding):
    """rho = 1, u = 0, no force: every field stays exactly zero in storage
    (rho - 1 = 0, j = 0) whatever the geometry."""
    for seed, per in [(1, (True, True)), (2, (False, False)), (3, (True, False))]:
        mask = wl.random_mask((131, 245), seed, 0.3, 0.1)
        d = binding.Domain(245, 131, per, (0.0, 0.0))
        d.set_geometry(mask)
        d.step(17)
        for a in d.get_state():
            assert not np.any(a)
        d.close()


def test_checkpoint_resume_is_bitwise(binding):
    p = wl.random_problem(300, 170, seed=8, periodic=(True, False))
    full = binding.Domain.from_problem(p)
    full.step(60)
    want = full.get_state()
    a = binding.Domain.from_problem(p)
    a.step(37)
    saved = a.get_state()
    b = binding.Domain(300, 170, p.periodic, p.force)
    b.set_geometry(p.mask)
    b.set_state(*saved)
    b.step(23)
    got = b.get_state()
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
    for dom in (full, a, b):
        dom.close()


def test_deterministic(binding):
    p = wl.porous(512, seed=3)
    outs = []
    for _ in range(2):
        d = binding.Domain.from_problem(p)
        d.step(301)
        outs.append((d.get_state(), d.residual()))
        d.close()
    for x, y in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(x, y)
    assert outs[0][1] == outs[1][1]


def test_unstable_state_is_reported(binding):
    """Failure detection on the host side: a state with a non-finite density,
    or a block of negative density large enough that the next step's output
    is still negative, makes the reduced step raise the sticky flag, which
    lbm_residual reports as LBM_E_UNSTABLE; loading a valid state clears it."""
    p = wl.random_problem(64, 40, seed=2, periodic=(True, True))
    cases = [("nan", (20, 30), np.nan, 3), ("negative block", (slice(15, 20), slice(40, 45)), -0.5, 1)]
    for name, where, value, nsteps in cases:
        d = binding.Domain.from_problem(p)
        mask = p.mask.copy()
        mask[where] = wl.FLUID
        d.set_geometry(mask)
        rho = p.rho.copy()
        rho[where] = value
        d.set_moments(rho, p.jx, p.jy)
        d.step(nsteps)
        with pytest.raises(binding.LbmError, match="UNSTABLE") as e:
            d.residual()
        assert e.value.status == binding.LBM_E_UNSTABLE, name
        d.set_moments(p.rho, p.jx, p.jy)
        d.step(3)
        res, mass = d.residual()
        assert np.isfinite(res), name
        d.close()


def test_copy_wait_timeout_is_reported(binding):
    """Failure detection without a fault: with a zero wait limit every wait
    of the step kernel for a staged row gives up at once; each warp then lets
    its copies in flight land (that drain keeps its one-second bound), raises
    the copy-timeout flag and stops.  lbm_residual reports LBM_E_CUDA with the
    timeout message, on a capturable stream (graph chunks) and on the default
    one; with the limit restored and the state loaded again, stepping gives
    the oracle's result."""
    import torch
    p = wl.random_problem(300, 170, seed=31, amp=0.02, periodic=(True, False))
    for stream in (None, torch.cuda.Stream()):
        d = binding.Domain.from_problem(p, stream=stream)
        d.step(40)          # graphs captured with the default limit
        d.set_copy_wait_ns(0)
        d.step(40)
        with pytest.raises(binding.LbmError, match="wait limit") as e:
            d.residual()
        assert e.value.status == binding.LBM_E_CUDA
        d.set_copy_wait_ns(10**9)
        d.set_moments(p.rho, p.jx, p.jy)
        d.step(20)
        res, mass = d.residual()
        assert np.isfinite(res)
        g = d.moments()
        d.close()
        o = oracle.run(p.mask, *p.state(), 20, p.periodic, p.force)
        for a, b in zip(g, o):
            assert np.abs(a - b).max() <= tolerance(0.02, 20)


def test_residual_matches_oracle(binding):
    p = wl.random_problem(200, 150, seed=6, amp=0.02, periodic=(False, True))
    d = binding.Domain.from_problem(p)
    d.step(40)
    res, mass = d.residual()
    d.close()
    o_prev = oracle.run(p.mask, *p.state(), 39, p.periodic, p.force)
    o_new = oracle.step(p.mask, *o_prev, p.periodic, p.force)
    r_ref, m_ref = oracle.residual(p.mask, o_prev, o_new)
    assert res == pytest.approx(r_ref, rel=1e-4)
    assert mass == pytest.approx(m_ref, rel=1e-7)


def test_independent_streams(binding):
    """Two domains stepped on two streams, interleaved, give the same bits as
    each run alone."""
    import torch
    p1 = wl.random_problem(333, 222, seed=11, periodic=(True, False))
    p2 = wl.cavity(300, 0.05)
    alone = []
    for p in (p1, p2):
        d = binding.Domain.from_problem(p)
        d.step(50)
        alone.append(d.get_state())
        d.close()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    d1 = binding.Domain.from_problem(p1, stream=s1)
    d2 = binding.Domain.from_problem(p2, stream=s2)
    for _ in range(10):
        d1.step(5)
        d2.step(5)
    for d, want in ((d1, alone[0]), (d2, alone[1])):
        for x, y in zip(d.get_state(), want):
            assert np.array_equal(x, y)
        d.close()
