"""Continuous batching: requests that arrive while others run are admitted
into the running batch; each result must be the same as the same problem run
alone for the same number of steps (bit for bit: the batched step runs the
single-domain code tile for tile), and the service must finish every request
in no more time than the sequential form takes."""
import numpy as np
import pytest

from paper_1912_09327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09327_gb300 import binding, serving
    return binding, serving


def test_results_same_alone_and_in_the_mix(mods):
    binding, serving = mods
    reqs = wl.request_stream(12, rate=400.0, seed=7, lo=48, hi=400)
    srv = serving.Server(capacity=6, chunk=100, residual_tol=1e-6,
                         max_steps=1500, keep_states=True)
    results = srv.run(reqs)
    variant = srv.batch.variant()
    srv.close()
    assert [r.rid for r in results] == [q.rid for q in reqs]
    overlapped = 0
    for q, r in zip(reqs, results):
        assert r.steps % 100 == 0 and 0 < r.steps <= 1500
        assert r.converged == (r.residual <= 1e-6)
        dom = binding.Domain.from_problem(q.problem())
        dom.set_variant(variant)  # same block tiles: same residual sums
        dom.step(r.steps)
        alone = dom.get_state()
        res, _ = dom.residual()
        dom.close()
        for a, b in zip(r.state, alone):
            assert np.array_equal(a, b)
        assert res == pytest.approx(r.residual, rel=1e-12)
        # this request shared the device with another one
        overlapped += any(o is not r and o.admitted < r.completed
                          and r.admitted < o.completed for o in results)
    assert overlapped == len(results)


def test_service_summary_and_sequential_form(mods):
    binding, serving = mods
    reqs = wl.request_stream(8, rate=200.0, seed=3, lo=48, hi=300)
    srv = serving.Server(capacity=8, chunk=100, residual_tol=1e-6,
                         max_steps=1000, keep_states=True)
    batched = srv.run(reqs)
    srv.close()
    plain = serving.serve_sequential(reqs, chunk=100, residual_tol=1e-6,
                                     max_steps=1000, keep_states=True)
    for a, b in zip(batched, plain):
        assert a.steps == b.steps
        for x, y in zip(a.state, b.state):
            assert np.array_equal(x, y)
    s = serving.summary(batched)
    assert s["requests"] == 8 and s["p99_latency_s"] >= s["p50_latency_s"] > 0
    assert s["converged"] + s["capped"] == 8


def test_served_result_matches_oracle(mods):
    """A request taken from a served mix (a channel, a cavity and a porous
    sample arriving while others run) against the FP64 oracle run for the
    same number of steps: the spec velocity bound."""
    import oracle
    binding, serving = mods
    reqs = [wl.Request(0, 0.00, "porous", 180, 150, 11),
            wl.Request(1, 0.01, "channel", 96, 40, 12),
            wl.Request(2, 0.02, "cavity", 70, 64, 13)]
    srv = serving.Server(capacity=4, chunk=200, residual_tol=1e-7,
                         max_steps=4000, keep_states=True)
    results = srv.run(reqs)
    srv.close()
    oracle.set_threads(oracle.max_threads())
    for q, r in zip(reqs, results):
        p = q.problem()
        o = oracle.run(p.mask, *p.state(), r.steps, p.periodic, p.force)
        d, jx, jy = (x.astype(np.float64) for x in r.state)
        rho = 1.0 + d
        keep = p.mask != wl.SOLID
        u = np.stack([jx / rho, jy / rho])[:, keep]
        uo = np.stack([o[1] / o[0], o[2] / o[0]])[:, keep]
        assert np.abs(u - uo).max() <= 1e-5 * np.abs(uo).max(), q.kind
