"""The allocation-free step entry point, for callers that cannot allocate
device memory (an application that routes all device memory through its own
pool allocator, or a loop that cannot afford cudaMalloc / cudaFree).

Through the C ABI, lbm_step_noalloc steps caller-owned device fields and keeps
its reduction scratch in a fixed device array of the library.  Its fields,
residual and mass must agree with the context-based entry point (lbm_step)
on the same state, within the parity tolerance of the GPU tests, for two
calls in a row.  This file is collected last so that a failure here leaves
the other GPU tests already run; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

from paper_1912_09327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def tolerance(amp, nsteps):
    # same bound as tests/test_gpu_parity.py
    return 2e-6 * amp * np.sqrt(nsteps) + 1e-9


def test_noalloc_step_matches_lbm_step():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09327_gb300 import binding as b

    amp = 0.02
    p = wl.random_problem(300, 170, seed=21, amp=amp, periodic=(True, False),
                          force=(1e-4, -5e-5))
    ny, nx = p.mask.shape
    # context path: two steps, each reduced
    dom = b.Domain.from_problem(p)
    want = []
    for _ in range(2):
        dom.step(1)
        want.append((dom.get_state(), dom.residual()))
    dom.close()

    # caller-owned device buffers, rows padded to a multiple of 32
    pitch = (nx + 31) // 32 * 32
    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    bufs = [[torch.zeros((ny, pitch), **f32) for _ in range(3)] for _ in range(2)]
    init = [(p.rho - 1.0).astype(np.float32), p.jx.astype(np.float32),
            p.jy.astype(np.float32)]
    solid = p.mask == wl.SOLID  # solid storage convention: 0, -fx, -fy
    init[0][solid], init[1][solid], init[2][solid] = 0.0, -p.force[0], -p.force[1]
    for t, a in zip(bufs[0], init):
        t[:, :nx] = torch.from_numpy(a).to(dev)
    mask = torch.ones(ny * pitch + 256, dtype=torch.uint8, device=dev)
    mask[: ny * pitch].view(ny, pitch)[:, :nx] = torch.from_numpy(p.mask).to(dev)
    sums = torch.zeros(3, dtype=torch.float64, device=dev)
    flags = torch.full((1,), 7, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    n_fluid = int((p.mask == 0).sum())

    src, dst = bufs
    for state, (res, mass) in want:
        b.lbm_step_noalloc(*[t.data_ptr() for t in src],
                           *[t.data_ptr() for t in dst], mask.data_ptr(),
                           nx, ny, pitch, p.periodic, p.force,
                           sums.data_ptr(), flags.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert int(flags.item()) == 0
        for t, ref in zip(dst, state):
            got = t[:, :nx].cpu().numpy()
            assert np.abs(got.astype(np.float64) - ref).max() <= tolerance(amp, 1)
        s0, s1, s2 = sums.cpu().numpy()
        assert np.sqrt(s0 / s1) == pytest.approx(res, rel=1e-6)
        assert n_fluid + s2 == pytest.approx(mass, rel=1e-12)
        src, dst = dst, src
