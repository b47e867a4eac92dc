"""16-bit storage of the moments (FP16 with power-of-two scaling, BF16),
FP32 arithmetic, stochastic or round-to-nearest rounding of the stored values.
A step from a state the 16-bit format represents exactly must equal the FP64
oracle's step from that same state up to one rounding of each output to the
format (half a unit in the last place to nearest, under one unit
stochastically; plus the FP32 arithmetic error); stochastic rounding keeps
the increments that round-to-nearest loses (closed form on a uniform periodic
box); over many steps the error against the oracle and against the analytic
Poiseuille profile is reported and bounded."""
import numpy as np
import pytest

import oracle
from paper_1912_09327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SCALE = {"f16": (1024.0, 64.0), "bf16": (1.0, 1.0)}
UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}   # unit roundoff of the format


def quantize(x, fmt, scale):
    """Round-to-nearest-even into the format, as the device stores it
    (double -> float32 -> 16 bit), returned as float64."""
    f = (np.asarray(x, np.float64) * scale).astype(np.float32)
    if fmt == "f16":
        q = f.astype(np.float16).astype(np.float32)
    else:
        bits = f.view(np.uint32).astype(np.uint64)
        bits = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16 << 16
        q = bits.astype(np.uint32).view(np.float32)
    return q.astype(np.float64) / scale


@pytest.fixture(scope="module")
def b():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09327_gb300 import binding
    return binding


@pytest.mark.parametrize("rounding", ["nearest", "stochastic"])
@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("nx,ny,per", [(300, 170, (True, False)),
                                       (61, 47, (False, True)),
                                       (500, 260, (True, True))])
def test_one_step_matches_oracle_to_format_rounding(b, fmt, nx, ny, per,
                                                    rounding):
    sd, sj = SCALE[fmt]
    p = wl.random_problem(nx, ny, seed=nx + ny, amp=0.02, periodic=per)
    R = 1.0 + quantize(p.rho - 1.0, fmt, sd)
    U = quantize(p.jx, fmt, sj)
    V = quantize(p.jy, fmt, sj)
    d = b.Domain(nx, ny, p.periodic, p.force, storage=fmt, rounding=rounding)
    d.set_geometry(p.mask)
    d.set_moments(R, U, V)
    d.step(1)
    g = d.moments()
    d.close()
    o = oracle.step(p.mask, R, U, V, p.periodic, p.force)
    # a unit in the last place is 2u: rounding to nearest errs by at most u,
    # stochastic rounding by less than 2u
    u = UNIT[fmt] * (2.0 if rounding == "stochastic" else 1.0)
    fluid = p.mask != wl.SOLID
    for got, want, sc in zip(g, o, (sd, sj, sj)):
        ref = want - 1.0 if sc == sd else want
        gg = got - 1.0 if sc == sd else got
        # one rounding to the format, the FP32 arithmetic, and the format's
        # smallest step near zero
        tol = u * np.abs(ref) + 2e-6 * 0.02 + 2.0 ** -24 / sc
        assert np.all(np.abs(gg - ref)[fluid] <= tol[fluid])


# Bounds: the measured errors with a margin (round to nearest is
# deterministic; the stochastic rounding draws its bits from the step count,
# so its errors repeat run to run too).  Measured, oracle / profile:
# f32 4.6e-6 / 1.6e-3, f16 nearest 0.180 / 0.181, bf16 nearest 0.608 / 0.609,
# f16 stochastic 1.3e-3 / 2.2e-3, bf16 stochastic 9.8e-3 / 5.9e-3.
@pytest.mark.parametrize("fmt,rounding,oracle_bound,profile_bound",
                         [("f32", "nearest", 1e-5, 1e-2),
                          ("f16", "nearest", 0.2, 0.2),
                          ("bf16", "nearest", 0.7, 0.7),
                          ("f16", "stochastic", 4e-3, 5e-3),
                          ("bf16", "stochastic", 3e-2, 2e-2)])
def test_channel_error_report(b, fmt, rounding, oracle_bound, profile_bound):
    """Channel 64 x 32, 5000 steps: relative velocity error against the FP64
    oracle and against the analytic parabola u = 3 f y (H - y).  Round-to-
    nearest 16-bit storage stalls once the per-step increments fall below
    half a unit in the last place; stochastic rounding does not."""
    p = wl.channel(64, 32, 0.01)
    d = b.Domain(64, 32, p.periodic, p.force, storage=fmt, rounding=rounding)
    d.set_geometry(p.mask)
    d.set_moments(p.rho, p.jx, p.jy)
    d.step(5000)
    R, U, V = d.moments()
    d.close()
    Ro, Uo, Vo = oracle.run(p.mask, *p.state(), 5000, p.periodic, p.force)
    u, uo = U / R, Uo / Ro
    err_oracle = np.abs(u - uo).max() / np.abs(uo).max()
    H = 31
    y = np.arange(1, 31)
    analytic = 3 * p.force[0] * y * (H - y)
    err_profile = (np.abs(u[1:-1, 0] - analytic).max() / analytic.max())
    print(fmt, rounding, "oracle", err_oracle, "profile", err_profile)
    assert np.isfinite(err_oracle) and err_oracle <= oracle_bound
    assert err_profile <= profile_bound


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_stochastic_rounding_keeps_small_increments(b, fmt):
    """Uniform periodic box, rho = 1, j = (0.01, 0), force F = (1e-6, 0): the
    method keeps the state uniform with j_n = j_0 + n F exactly (every
    equilibrium sums back to the node's own moments).  F is below half a unit
    in the last place of j in both formats, so round-to-nearest never moves;
    stochastic rounding tracks j_0 + n F on average (the mean of N nodes
    carries sqrt(n / N) units of noise, far below the 2 % bound)."""
    nx, ny, n, F, j0 = 512, 256, 1000, 1e-6, 0.01
    mask = np.zeros((ny, nx), np.uint8)
    rho = np.ones((ny, nx))
    jx = np.full((ny, nx), j0)
    jy = np.zeros((ny, nx))
    means = {}
    for rounding in ("nearest", "stochastic"):
        d = b.Domain(nx, ny, (True, True), (F, 0.0), storage=fmt,
                     rounding=rounding)
        d.set_geometry(mask)
        d.set_moments(rho, jx, jy)
        d.step(n)
        R, U, V = d.moments()
        d.close()
        means[rounding] = (U.mean(), V.mean(), (R - 1.0).mean())
    # j0 is stored rounded; the drift is what matters
    jq = quantize(np.array([j0]), fmt, SCALE[fmt][1])[0]
    assert abs(means["nearest"][0] - jq) < 0.1 * n * F
    assert means["stochastic"][0] - jq == pytest.approx(n * F, rel=0.02)
    assert abs(means["stochastic"][1]) < 0.02 * n * F
    assert abs(means["stochastic"][2]) < 1e-5


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_stochastic_rounding_is_reproducible_and_resumable(b, fmt):
    """The random bits come from (column, row, field, step count): two runs
    agree bit for bit, and a run saved (state and step count) and resumed in
    a new context continues bit for bit."""
    p = wl.random_problem(333, 141, seed=9, amp=0.02, periodic=(True, False))

    def make():
        d = b.Domain(333, 141, p.periodic, p.force, storage=fmt)
        d.set_geometry(p.mask)
        d.set_moments(p.rho, p.jx, p.jy)
        return d

    runs = []
    for _ in range(2):
        d = make()
        d.step(40)
        runs.append(d.get_state())
        assert d.step_count() == 40
        d.close()
    for x, y in zip(*runs):
        assert np.array_equal(x.view(np.uint16), y.view(np.uint16))
    d = make()
    d.step(17)
    saved, steps = d.get_state(), d.step_count()
    d.close()
    e = make()
    e.set_state(*saved)
    e.set_step_count(steps)
    e.step(23)
    resumed = e.get_state()
    e.close()
    for x, y in zip(resumed, runs[0]):
        assert np.array_equal(x.view(np.uint16), y.view(np.uint16))


def test_change_since_snapshot(b):
    """The span change (lbm_snapshot / lbm_change_since) is the FP64 mean
    relative velocity change per step, as computed on the host from the two
    states; on the FP16 channel at its steady state the per-step residual
    sits at the rounding noise while the change over 10000 steps falls two
    orders below it, so a 16-bit solve has a convergence test that fires."""
    p = wl.channel(64, 32, 0.01)
    d = b.Domain.from_problem(p, storage="f16")
    d.step(20000)
    res, _ = d.residual()
    snap = d.snapshot()
    R0, U0, V0 = d.moments()
    d.step(10000)
    ch = d.change_since(snap, 10000)
    R1, U1, V1 = d.moments()
    d.close()
    fluid = p.mask == 0
    num = (((U1 / R1 - U0 / R0) ** 2 + (V1 / R1 - V0 / R0) ** 2)[fluid]).sum()
    den = (((U1 / R1) ** 2 + (V1 / R1) ** 2)[fluid]).sum()
    assert ch == pytest.approx(np.sqrt(num / den) / 10000, rel=1e-6)
    assert res > 1e-4              # the per-step residual: rounding noise
    assert ch < res / 100          # the span change: below it by far
