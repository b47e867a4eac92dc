"""The allocation-free step entry point, for callers that cannot allocate
device memory (an application that routes all device memory through its own
pool allocator, or a loop that cannot afford cudaMalloc / cudaFree).

Through the C ABI, lbm_step_noalloc steps caller-owned device fields and keeps
its reduction scratch in a fixed device array of the library.  It launches
the same kernel with the same tile variant as the context-based entry point
(lbm_step) and sums the same partials in the same order, so on the same state
its fluid and fixed nodes, residual sums and mass agree with lbm_step's bit
for bit, for two calls in a row, for a smaller domain after a larger one
(stale partials or a stale flag left in the shared array would show there),
and whatever the caller leaves in its solid nodes.  A domain needing more
thread blocks than the array serves is rejected before anything runs.  This
file is collected last so that a failure here leaves the other GPU tests
already run; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

from paper_1912_09327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09327_gb300 import binding as b
    return torch, b


def context_steps(b, p, nsteps):
    """States (exact storage) and (residual, mass) after each of nsteps
    reduced steps through the context path."""
    dom = b.Domain.from_problem(p)
    out = []
    for _ in range(nsteps):
        dom.step(1)
        out.append((dom.get_state(), dom.residual()))
    dom.close()
    return out


class Buffers:
    """Caller-owned device fields (two copies), node types, sums and flag,
    rows padded to a multiple of 32 nodes.  Solid nodes get `junk`: the step
    never reads what a solid node holds."""

    def __init__(self, torch, p, junk):
        ny, nx = p.mask.shape
        self.nx, self.ny = nx, ny
        self.pitch = (nx + 31) // 32 * 32
        dev = torch.device("cuda")
        f32 = dict(dtype=torch.float32, device=dev)
        self.f = [[torch.full((ny, self.pitch), np.nan, **f32)
                   for _ in range(3)] for _ in range(2)]
        init = [(p.rho - 1.0).astype(np.float32), p.jx.astype(np.float32),
                p.jy.astype(np.float32)]
        solid = p.mask == wl.SOLID
        for k, a in enumerate(init):
            a[solid] = junk[k]
            self.f[0][k][:, :nx] = torch.from_numpy(a).to(dev)
        self.mask = torch.ones(ny * self.pitch + 256, dtype=torch.uint8,
                               device=dev)
        self.mask[: ny * self.pitch].view(ny, self.pitch)[:, :nx] = \
            torch.from_numpy(p.mask).to(dev)
        self.sums = torch.full((3,), np.nan, dtype=torch.float64, device=dev)
        self.flags = torch.full((1,), 7, dtype=torch.int32, device=dev)


def noalloc_step(torch, b, buf, p, src, dst):
    stream = torch.cuda.current_stream()
    b.lbm_step_noalloc(*[t.data_ptr() for t in buf.f[src]],
                       *[t.data_ptr() for t in buf.f[dst]],
                       buf.mask.data_ptr(), buf.nx, buf.ny, buf.pitch,
                       p.periodic, p.force, buf.sums.data_ptr(),
                       buf.flags.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()


def check_against_context(torch, b, p, junk, nsteps=2):
    want = context_steps(b, p, nsteps)
    buf = Buffers(torch, p, junk)
    keep = p.mask != wl.SOLID
    n_fluid = int((p.mask == wl.FLUID).sum())
    src, dst = 0, 1
    for state, (res, mass) in want:
        noalloc_step(torch, b, buf, p, src, dst)
        assert int(buf.flags.item()) == 0
        for t, ref in zip(buf.f[dst], state):
            got = t[:, : buf.nx].cpu().numpy()
            assert np.array_equal(got[keep].view(np.uint32),
                                  ref[keep].view(np.uint32))
        s0, s1, s2 = buf.sums.cpu().numpy()
        assert np.sqrt(s0 / s1) == res
        assert n_fluid + s2 == mass
        src, dst = dst, src


def test_noalloc_step_matches_lbm_step(env):
    """Two calls in a row on a random walled/periodic domain with force,
    with NaN in every solid node of the caller's fields."""
    torch, b = env
    p = wl.random_problem(300, 170, seed=21, amp=0.02, periodic=(True, False),
                          force=(1e-4, -5e-5))
    check_against_context(torch, b, p, junk=(np.nan, np.nan, np.nan))


def test_noalloc_smaller_domain_after_larger(env):
    """A large domain then a small one: the second call must read none of
    the first call's partials and must start from a cleared flag (here after
    a call that raised it: a NaN in a fluid node)."""
    torch, b = env
    big = wl.random_problem(1000, 700, seed=5, amp=0.02,
                            periodic=(False, True))
    buf = Buffers(torch, big, junk=(1e30, -1e30, 3.0))
    buf.f[0][0][10, 10] = float("nan")
    big.mask[10, 10] = wl.FLUID
    buf.mask[10 * buf.pitch + 10] = wl.FLUID
    noalloc_step(torch, b, buf, big, 0, 1)
    assert int(buf.flags.item()) & 1  # instability raised for the big one
    small = wl.random_problem(97, 61, seed=6, amp=0.02, periodic=(True, True),
                              force=(2e-5, 1e-5))
    check_against_context(torch, b, small, junk=(7.0, 7.0, -7.0))


def test_noalloc_rejects_oversized_domain(env):
    """A domain needing more thread blocks than the static scratch serves
    is refused with LBM_E_INVAL before any launch (the buffers passed are
    small, valid device memory that nothing touches)."""
    torch, b = env
    n = 1 << 20
    dev = torch.device("cuda")
    f = torch.zeros(64, dtype=torch.float32, device=dev)
    m = torch.zeros(64, dtype=torch.uint8, device=dev)
    sums = torch.zeros(3, dtype=torch.float64, device=dev)
    flags = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(b.LbmError) as e:
        b.lbm_step_noalloc(*[f.data_ptr()] * 6, m.data_ptr(), n, n, n,
                           (True, True), (0.0, 0.0), sums.data_ptr(),
                           flags.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    assert e.value.status == b.LBM_E_INVAL
    torch.cuda.synchronize()
    assert not torch.any(f) and not torch.any(sums)
