"""Batched stepping (one launch per step for many domains) against stepping
each domain alone and against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1912_09327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09327_gb300 import binding
    return binding


def mixed_problems(count, seed=0, lo=20, hi=700):
    """Seeded mix of channels, cavities, porous samples and random domains
    with log-uniform side lengths."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx, ny = (int(round(v)) for v in np.exp(rng.uniform(np.log(lo), np.log(hi), 2)))
        kind = i % 4
        if kind == 0:
            p = wl.channel(nx, max(ny, 5), 0.01)
        elif kind == 1:
            p = wl.cavity(nx, 0.1, ny=max(ny, 4))
        elif kind == 2:
            p = wl.porous(max(nx, 64), seed=i, r_min=3, r_max=8,
                          ny=max(ny, 64), fx=1e-4)
        else:
            p = wl.random_problem(nx, ny, seed=i, periodic=(bool(i & 4), bool(i & 8)))
        out.append(p)
    return out


def states(doms):
    return [d.get_state() for d in doms]


@pytest.mark.parametrize("nsteps", [1, 2, 37])
def test_batch_equals_each_alone(b, nsteps):
    """Same states bit for bit; with the batch's tile variant on the
    single-domain path as well (same block tiles, same partial sums), the same
    residual and mass bit for bit too."""
    probs = mixed_problems(10, seed=nsteps)
    import torch
    stream = torch.cuda.Stream()  # a capturable stream: graph chunks are used
    batch = b.Batch(len(probs), 100000, stream=stream)
    alone = []
    for p in probs:
        d = b.Domain.from_problem(p)
        d.set_variant(batch.variant())
        d.step(nsteps)
        alone.append((d.get_state(), d.residual()))
        d.close()
    doms = [b.Domain.from_problem(p, stream=stream) for p in probs]
    for d in doms:
        batch.add(d)
    batch.step(nsteps)
    for d, (want, (res, mass)) in zip(doms, alone):
        for x, y in zip(d.get_state(), want):
            assert np.array_equal(x, y)
        r2, m2 = d.residual()
        assert r2 == pytest.approx(res, rel=1e-12, abs=1e-300)
        assert m2 == pytest.approx(mass, rel=1e-12)
    batch.close()


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_batch_stochastic_rounding_equals_alone(b, fmt):
    """16-bit storage with stochastic rounding: a member's random bits follow
    its own step count (the batch clock advanced by each launch, offset per
    member), so batched steps, graph chunks included, give every member the
    state it reaches alone, bit for bit; also after a member stepped on its
    own in between."""
    probs = mixed_problems(6, seed=21)
    import torch
    stream = torch.cuda.Stream()
    alone = []
    for p in probs:
        d = b.Domain.from_problem(p, storage=fmt)
        d.step(5)
        d.step(37)
        alone.append(d.get_state())
        d.close()
    doms = [b.Domain.from_problem(p, stream=stream, storage=fmt) for p in probs]
    batch = b.Batch(len(doms), 100000, stream=stream)
    doms[0].step(5)                 # member 0 on its own first: 5
    slots = [batch.add(d) for d in doms]
    batch.step(5)                   # member 0 at 10, the others at 5
    batch.remove(slots[0])
    batch.step(32)                  # the others at 37 (graph chunks)
    doms[0].step(27)                # member 0 on its own to 37
    batch.add(doms[0])
    batch.step(5)                   # everyone at 42
    for d, want in zip(doms, alone):
        assert d.step_count() == 42
        for x, y in zip(d.get_state(), want):
            assert np.array_equal(x.view(np.uint16), y.view(np.uint16))
    batch.close()


def test_batch_variants_are_identical_and_autotune(b):
    probs = mixed_problems(6, seed=11)
    import torch
    stream = torch.cuda.current_stream()
    results = []
    for v in range(b.lbm_variant_count()):
        doms = [b.Domain.from_problem(p, stream=stream) for p in probs]
        batch = b.Batch(len(doms), 100000, stream=stream)
        for d in doms:
            batch.add(d)
        batch.set_variant(v)
        batch.step(21)
        results.append(states(doms))
        batch.close()
    for r in results[1:]:
        for sa, sb in zip(results[0], r):
            for x, y in zip(sa, sb):
                assert np.array_equal(x, y)
    # autotune: real steps, every variant timed, the fastest kept
    doms = [b.Domain.from_problem(p, stream=stream) for p in probs]
    batch = b.Batch(len(doms), 100000, stream=stream)
    for d in doms:
        batch.add(d)
    chosen, ms = batch.autotune(4)
    assert 0 <= chosen < b.lbm_variant_count()
    assert all(t > 0 for t in ms) and ms[chosen] == min(ms)
    ref = [b.Domain.from_problem(p, stream=stream) for p in probs]
    for d in ref:
        d.step((4 + 2) * b.lbm_variant_count())
    for d, r in zip(doms, ref):
        for x, y in zip(d.get_state(), r.get_state()):
            assert np.array_equal(x, y)
    batch.close()


def test_batch_membership_changes(b):
    probs = mixed_problems(5, seed=3)
    import torch
    stream = torch.cuda.current_stream()
    doms = [b.Domain.from_problem(p, stream=stream) for p in probs]
    batch = b.Batch(4, 100000, stream=stream)
    slots = [batch.add(d) for d in doms[:4]]
    with pytest.raises(b.LbmError):
        batch.add(doms[4])            # full
    batch.step(5)
    batch.remove(slots[1])            # doms[1] leaves after 5 steps
    batch.add(doms[4])                # doms[4] joins at 0 steps
    batch.step(6)
    counts = [11, 5, 11, 11, 6]
    for d, p, n in zip(doms, probs, counts):
        ref = b.Domain.from_problem(p, stream=stream)
        ref.step(n)
        for x, y in zip(d.get_state(), ref.get_state()):
            assert np.array_equal(x, y)
    batch.close()


def test_batch_clean_tiles_run_last_and_equal_alone(b):
    """A batch whose kernel carries the clean-tile code, with members that
    have clean warp tiles (a 600 x 600 cavity, a 700 x 300 channel) beside
    small ones, orders its work list by tile kind (general tiles first);
    every member still reaches the state it reaches alone, bit for bit,
    also after a member leaves and the list is rebuilt, and after a member's
    node types change (its flags are computed again)."""
    import torch
    stream = torch.cuda.current_stream()
    dual = [v for v in range(b.lbm_variant_count())
            if b.lbm_variant_has_clean_code(v)][0]
    tx, ty, _ = b.lbm_variant_tile(dual)
    probs = [wl.cavity(600, 0.1), wl.channel(700, 300, 0.01), wl.cavity(40, 0.1),
             wl.porous(100, seed=2, r_min=3, r_max=8, ny=90, fx=1e-4)]
    doms = [b.Domain.from_problem(p, stream=stream) for p in probs]
    batch = b.Batch(len(doms), 100000, stream=stream)
    slots = [batch.add(d) for d in doms]
    batch.set_variant(dual)
    batch.step(15)
    batch.remove(slots[2])
    batch.step(10)
    # new node types for the channel: a solid block in its middle
    mask = probs[1].mask.copy()
    mask[100:140, 300:340] = wl.SOLID
    doms[1].set_geometry(mask)
    doms[1].set_moments(probs[1].rho, probs[1].jx, probs[1].jy)
    batch.step(7)
    counts = [32, 7, 15, 32]
    for i, (d, p, n) in enumerate(zip(doms, probs, counts)):
        ref = b.Domain.from_problem(p, stream=stream)
        if i == 1:
            ref.set_geometry(mask)
            ref.set_moments(p.rho, p.jx, p.jy)
        ref.step(n)
        for x, y in zip(d.get_state(), ref.get_state()):
            assert np.array_equal(x, y), i
        ref.close()
    batch.close()
    for d in doms:
        d.close()


def test_batch_member_matches_oracle(b):
    p = wl.random_problem(300, 170, seed=5, periodic=(True, False))
    q = wl.cavity(257, 0.1, ny=133)
    import torch
    stream = torch.cuda.current_stream()
    doms = [b.Domain.from_problem(x, stream=stream) for x in (p, q)]
    batch = b.Batch(2, 10000, stream=stream)
    for d in doms:
        batch.add(d)
    batch.step(20)
    for d, x in zip(doms, (p, q)):
        o = oracle.run(x.mask, *x.state(), 20, x.periodic, x.force)
        g = d.moments()
        fluid = x.mask != wl.SOLID
        amp = max(np.abs(x.rho - 1).max(), np.abs(x.jx).max(), 1e-3)
        for a_, b_ in zip(g, o):
            assert np.abs(a_ - b_)[fluid].max() <= 2e-6 * amp * np.sqrt(20) + 1e-9
    batch.close()


def velocity_error(a, b):
    ua = np.stack([a[1] / a[0], a[2] / a[0]])
    ub = np.stack([b[1] / b[0], b[2] / b[0]])
    return np.abs(ua - ub).max() / np.abs(ub).max()


def test_batch_mix512_sample_matches_oracle(b):
    """The batched configuration itself: all 512 domains of the seeded mix
    (channel / cavity / porous thirds, sides log-uniform in [64, 1024]) in
    one batch with the autotuner's tile variant, 2000 steps, FP32 storage
    with stochastic rounding of the momentum; a seeded sample of 16 members
    (the largest of each kind among them included) is compared node by node
    with the oracle's 2000 steps, at the 1e-5 velocity bound.  (Rounded to
    nearest, FP32 storage alone drifts past that bound on the slowly
    accelerating channels of the mix: tests/test_fp32_storage_floor.py.)"""
    import torch
    oracle.set_threads(oracle.max_threads())
    probs = wl.batch_mix(512, seed=0)
    rng = np.random.default_rng(512)
    pick = set(int(i) for i in rng.choice(len(probs), 13, replace=False))
    for k in range(3):   # the largest domain of each kind
        same = [i for i in range(len(probs)) if i % 3 == k]
        pick.add(max(same, key=lambda i: probs[i].mask.size))
    pick = sorted(pick)[:16]
    stream = torch.cuda.Stream()
    doms = [b.Domain.from_problem(p, stream=stream, rounding="stochastic")
            for p in probs]
    tiles = sum(b.lbm_tile_count(p.mask.shape[1], p.mask.shape[0])
                for p in probs)
    batch = b.Batch(len(doms), tiles, stream=stream)
    for d in doms:
        batch.add(d)
    batch.autotune(2)          # real steps: the members start again below
    for d, p in zip(doms, probs):
        d.set_moments(p.rho, p.jx, p.jy)
    batch.step(2000)
    res, _, status = batch.residuals()
    assert all(s == b.LBM_OK for s in status[: len(doms)])
    got = {i: doms[i].moments() for i in pick}
    batch.close()
    for d in doms:
        d.close()
    # the same mix in 16-bit storage (stochastic rounding)
    got16 = {}
    for fmt in ("f16", "bf16"):
        doms = [b.Domain.from_problem(p, stream=stream, storage=fmt)
                for p in probs]
        batch = b.Batch(len(doms), tiles, stream=stream)
        for d in doms:
            batch.add(d)
        batch.step(2000)
        got16[fmt] = {i: doms[i].moments() for i in pick}
        batch.close()
        for d in doms:
            d.close()
    worst = {"f32": 0.0, "f16": 0.0, "bf16": 0.0}
    for i in pick:
        p = probs[i]
        o = oracle.run(p.mask, *p.state(), 2000, p.periodic, p.force)
        g = got[i]
        err = velocity_error(g, o)
        assert err <= 1e-5, (i, p.name, p.mask.shape, err)
        assert np.abs(g[0] - o[0]).max() <= 1e-5, (i, p.name)
        worst["f32"] = max(worst["f32"], err)
        for fmt in ("f16", "bf16"):
            worst[fmt] = max(worst[fmt], velocity_error(got16[fmt][i], o))
    print("batch mix sample x 2000, worst max|du|/max|u|:", worst)
    assert worst["f16"] <= 4e-3 and worst["bf16"] <= 4e-2, worst
