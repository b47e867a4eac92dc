"""The seeded input recipes: each generator builds the geometry, force and
initial state its configuration states (channel and cavity of Section 3 and
Appendix A, the porous sample, the bandwidth-sweep box, the batch and request
mixes)."""
import numpy as np
import pytest

from paper_1912_09327_gb300 import workloads as wl


def test_channel_recipe():
    p = wl.channel(64, 32, 0.01)
    assert p.mask.shape == (32, 64) and p.periodic == (True, False)
    assert np.all(p.mask[0] == wl.SOLID) and np.all(p.mask[-1] == wl.SOLID)
    assert np.all(p.mask[1:-1] == wl.FLUID)
    # f = 8 nu u_max / H^2 with nu = 1/6, H = 31
    assert p.force == pytest.approx((8.0 / 6.0 * 0.01 / 31 ** 2, 0.0), rel=1e-14)
    assert p.force[0] == pytest.approx(1.38744e-5, rel=1e-5)
    assert np.all(p.rho == 1.0) and not p.jx.any() and not p.jy.any()


def test_cavity_recipe():
    n = 40
    p = wl.cavity(n, 0.1)
    m = p.mask
    assert p.periodic == (False, False) and p.force == (0.0, 0.0)
    assert np.all(m[:, 0] == wl.SOLID) and np.all(m[:, -1] == wl.SOLID)
    assert np.all(m[0, :] == wl.SOLID)
    assert m[-1, 0] == wl.SOLID and m[-1, -1] == wl.SOLID   # top corners
    assert np.all(m[-1, 1:-1] == wl.FIXED)
    assert np.all(m[1:-1, 1:-1] == wl.FLUID)
    assert np.all(p.jx[-1, 1:-1] == 0.1) and np.all(p.rho == 1.0)
    assert not p.jx[:-1].any() and not p.jy.any()


def test_porous_recipe():
    p = wl.porous(256, seed=3, r_min=4, r_max=10)
    assert p.periodic == (True, True) and p.force == (1e-5, 0.0)
    frac = (p.mask == wl.SOLID).mean()
    assert 0.30 <= frac < 0.33
    assert p.meta["solid_fraction"] == pytest.approx(frac)
    assert 8.0 <= p.meta["mean_diameter"] <= 20.0
    assert set(np.unique(p.mask)) <= {wl.FLUID, wl.SOLID}
    # the same seed gives the same sample
    assert np.array_equal(p.mask, wl.porous(256, seed=3, r_min=4, r_max=10).mask)


def test_sweep_box_is_periodic_random_field():
    p = wl.periodic_box_tiled(1024, seed=1, tile=256)
    assert p.periodic == (True, True) and not p.mask.any()
    for a in (p.rho, p.jx, p.jy):
        assert a.shape == (1024, 1024)
        assert np.array_equal(a[:256, :256], a[256:512, 768:])
    d = p.rho - 1.0
    assert abs(d.std() - 1e-3) < 1e-4 and abs(d.mean()) < 1e-4
    small = wl.periodic_box_tiled(100, tile=512)
    assert small.rho.shape == (100, 100)


def test_batch_mix_recipe():
    probs = wl.batch_mix(24, seed=0)
    assert [p.name for p in probs[:3]] == ["channel", "cavity", "porous"]
    for p in probs:
        ny, nx = p.mask.shape
        assert 64 <= nx <= 1024 and 64 <= ny <= 1024


def test_request_stream_recipe():
    reqs = wl.request_stream(4000, rate=200.0, seed=0)
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert np.all(gaps > 0)
    assert gaps.mean() == pytest.approx(1 / 200.0, rel=0.05)
    assert gaps.std() == pytest.approx(1 / 200.0, rel=0.1)   # exponential
    assert all(64 <= r.nx <= 2048 and 64 <= r.ny <= 2048 for r in reqs)
    kinds = [r.kind for r in reqs]
    for k in wl.KINDS:
        assert kinds.count(k) / len(kinds) == pytest.approx(1 / 3, abs=0.04)


def test_serving_admission_order():
    """Smallest first, earliest among equals; the oldest first once it has
    waited longer than max_wait; plain arrival order under "fifo"."""
    from paper_1912_09327_gb300 import serving
    R = wl.Request
    w = [R(0, 0.00, "cavity", 900, 900, 0), R(1, 0.01, "channel", 64, 80, 1),
         R(2, 0.02, "porous", 64, 80, 2), R(3, 0.03, "cavity", 300, 64, 3)]
    assert serving.select_next(w, 0.1).rid == 1
    assert serving.select_next(w, 0.1, policy="fifo").rid == 0
    assert serving.select_next(w, 2.5, max_wait=2.0).rid == 0
    assert serving.select_next(w[2:], 2.5, max_wait=2.0).rid == 2
    assert serving.select_next([], 0.0) is None


def test_serving_batch_variant_model():
    """The service's tile variant for a batch: least padded tile work.  Many
    64 x 64 domains fit the 16-row warp tiles (one 120 x 64 block tile each);
    one 4096^2 domain wastes little in the tall default tiles, which march
    fewer halo rows."""
    from paper_1912_09327_gb300 import binding, serving
    small = serving.choose_batch_variant([(64, 64)] * 20)
    tx, ty, cols = binding.lbm_variant_tile(small)
    assert ty == 64 and cols == 4
    big = serving.choose_batch_variant([(4096, 4096)])
    assert binding.lbm_variant_tile(big)[1] == 256
    # of the two variants with those tiles, the one with the clean-tile code
    assert binding.lbm_variant_has_clean_code(big)
    assert 0 <= serving.choose_batch_variant([(1, 1)]) < binding.lbm_variant_count()
