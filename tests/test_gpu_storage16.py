"""16-bit storage of the moments (FP16 with power-of-two scaling, BF16),
FP32 arithmetic.  A step from a state the 16-bit format represents exactly
must equal the FP64 oracle's step from that same state up to one rounding of
each output to the format (plus the FP32 arithmetic error); over many steps
the error against the oracle and against the analytic Poiseuille profile is
reported (and bounded loosely)."""
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


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("nx,ny,per", [(300, 170, (True, False)),
                                       (61, 47, (False, True)),
                                       (500, 260, (True, True))])
def test_one_step_matches_oracle_to_format_rounding(b, fmt, nx, ny, per):
    sd, sj = SCALE[fmt]
    p = wl.random_problem(nx, ny, seed=nx + ny, amp=0.02, periodic=per)
    R = 1.0 + quantize(p.rho - 1.0, fmt, sd)
    U = quantize(p.jx, fmt, sj)
    V = quantize(p.jy, fmt, sj)
    d = b.Domain(nx, ny, p.periodic, p.force, storage=fmt)
    d.set_geometry(p.mask)
    d.set_moments(R, U, V)
    d.step(1)
    g = d.moments()
    d.close()
    o = oracle.step(p.mask, R, U, V, p.periodic, p.force)
    u = UNIT[fmt]
    fluid = p.mask != wl.SOLID
    for got, want, sc in zip(g, o, (sd, sj, sj)):
        ref = want - 1.0 if sc == sd else want
        gg = got - 1.0 if sc == sd else got
        # one rounding to the format, the FP32 arithmetic, and the format's
        # smallest step near zero
        tol = u * np.abs(ref) + 2e-6 * 0.02 + 2.0 ** -24 / sc
        assert np.all(np.abs(gg - ref)[fluid] <= tol[fluid])


@pytest.mark.parametrize("fmt,oracle_bound,profile_bound",
                         [("f32", 1e-5, 1e-2), ("f16", 0.2, 0.25),
                          ("bf16", 1.0, 1.0)])
def test_channel_error_report(b, fmt, oracle_bound, profile_bound):
    """Channel 64 x 32, 5000 steps: relative velocity error against the FP64
    oracle and against the analytic parabola u = 3 f y (H - y)."""
    p = wl.channel(64, 32, 0.01)
    d = b.Domain(64, 32, p.periodic, p.force, storage=fmt)
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
    print(fmt, "oracle", err_oracle, "profile", err_profile)
    assert np.isfinite(err_oracle) and err_oracle <= oracle_bound
    assert err_profile <= profile_bound
