"""Host-side checks of the C ABI library (no GPU needed): it loads, exports
every function include/lbmtau1.h declares, sizes its workspace after the
paper's storage model, and validates arguments before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbmtau1.h")


@pytest.fixture(scope="module")
def b():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09327_gb300 import binding
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(b):
    names = declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(b.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_follows_storage_model(b):
    """Eq. (LBMTau1memory): 2 N_f c = 24 bytes per node for the two copies of
    (rho, u_x, u_y) in FP32, against (2Q + N_f) c = 84 for the standard
    algorithm (Eq. lbmmemory); golden values from Section 4."""
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "memory_model.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            gold[k] = int(v)
    Q, Nf, c = gold["Q"], gold["N_f"], gold["bytes_per_number_float"]
    assert 2 * Nf * c == gold["lbmtau1_bytes_per_node"]
    assert (2 * Q + Nf) * c == gold["standard_lbm_bytes_per_node"]
    # large domain: fields (24 B) + node type (1 B) + bounded extras
    n = 16384
    ws = b.lbm_workspace_bytes(b.make_params(n, n))
    per_node = ws / (n * n)
    assert gold["lbmtau1_bytes_per_node"] + 1 <= per_node < 25.2
    # the paper's 1000 x 1000 example: 24 MB of fields (rows padded to 1024)
    ws1000 = b.lbm_workspace_bytes(b.make_params(1000, 1000))
    fields = 6 * 4 * 1024 * 1000
    assert fields / 1e6 == pytest.approx(gold["cavity_1000_lbmtau1_MB"], rel=0.03)
    assert ws1000 >= fields + 1024 * 1000


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=0), dict(nx=-3),
                                 dict(storage=7), dict(rounding=3), dict(rounding=-1),
                                 dict(fx=float("nan")), dict(sc_g=float("inf")),
                                 dict(sc_g=-5.0, storage=1),
                                 dict(sc_g=-5.0, storage=2)])
def test_invalid_params(b, bad):
    p = b.make_params(10, 10)
    for k, v in bad.items():
        setattr(p, k, v)
    assert b.lbm_workspace_bytes(p) == 0
    ctx = ctypes.c_void_p()
    st = b._lib.lbm_create(ctypes.byref(p), ctypes.c_void_p(1 << 20), 1 << 40,
                           None, ctypes.byref(ctx))
    assert st == b.LBM_E_INVAL and not ctx.value


def test_create_validates_workspace(b):
    p = b.make_params(100, 50)
    need = b.lbm_workspace_bytes(p)
    ctx = ctypes.c_void_p()
    create = b._lib.lbm_create
    assert create(ctypes.byref(p), None, need, None, ctypes.byref(ctx)) == b.LBM_E_WORKSPACE
    assert create(ctypes.byref(p), ctypes.c_void_p(4096 + 8), need, None,
                  ctypes.byref(ctx)) == b.LBM_E_WORKSPACE
    assert create(ctypes.byref(p), ctypes.c_void_p(4096), need - 1, None,
                  ctypes.byref(ctx)) == b.LBM_E_WORKSPACE
    assert create(ctypes.byref(p), ctypes.c_void_p(4096), need, None, None) == b.LBM_E_INVAL


def test_call_order_and_arguments_checked_on_host(b):
    """A context over a never-dereferenced aligned address: every call below
    fails its host-side checks before touching the device."""
    p = b.make_params(20, 10, (True, False), (1e-5, 0))
    ctx = b.lbm_create(p, 1 << 20, b.lbm_workspace_bytes(p))
    try:
        lib = b._lib
        assert lib.lbm_step(ctx, 5) == b.LBM_E_STATE
        assert "geometry" in b.lbm_last_error(ctx)
        assert lib.lbm_step(ctx, -1) == b.LBM_E_INVAL
        assert lib.lbm_residual(ctx, None, None) == b.LBM_E_STATE
        assert lib.lbm_moments(ctx, None, None, None) == b.LBM_E_INVAL
        assert lib.lbm_get_state(ctx, None, None, None) == b.LBM_E_INVAL
        assert lib.lbm_set_geometry(ctx, None) == b.LBM_E_INVAL
        bad = np.zeros((10, 20), np.uint8)
        bad[3, 4] = 3
        assert lib.lbm_set_geometry(ctx, bad.ctypes.data) == b.LBM_E_INVAL
        assert "type 3" in b.lbm_last_error(ctx)
        z = np.zeros(200)
        assert lib.lbm_set_moments(ctx, z.ctypes.data, z.ctypes.data,
                                   z.ctypes.data) == b.LBM_E_STATE
        nv = b.lbm_variant_count()
        assert nv >= 1
        assert lib.lbm_set_variant(ctx, nv) == b.LBM_E_INVAL
        assert lib.lbm_set_variant(ctx, -2) == b.LBM_E_INVAL
        for v in range(nv):
            assert lib.lbm_set_variant(ctx, v) == b.LBM_OK
            assert b.lbm_variant(ctx) == v
        assert lib.lbm_set_variant(ctx, -1) == b.LBM_OK
        # the staged-row wait limit: 0 .. 1 s
        assert lib.lbm_set_copy_wait_ns(ctx, -1) == b.LBM_E_INVAL
        assert lib.lbm_set_copy_wait_ns(ctx, 10**9 + 1) == b.LBM_E_INVAL
        assert lib.lbm_set_copy_wait_ns(ctx, 0) == b.LBM_OK
        assert lib.lbm_set_copy_wait_ns(ctx, 10**9) == b.LBM_OK
        assert lib.lbm_set_copy_wait_ns(None, 0) == b.LBM_E_INVAL
        # the step count that seeds stochastic rounding
        assert b.lbm_step_count(ctx) == 0
        b.lbm_set_step_count(ctx, 12345)
        assert b.lbm_step_count(ctx) == 12345
        assert lib.lbm_set_step_count(ctx, -1) == b.LBM_E_INVAL
        assert lib.lbm_step_count(ctx, None) == b.LBM_E_INVAL
        # tile counts: each variant's grid, and the bound over all of them
        counts = [b.lbm_tile_count(1000, 700, v) for v in range(nv)]
        assert all(c >= 1 for c in counts)
        assert b.lbm_tile_count(1000, 700) == max(counts)
        assert b.lbm_tile_count(120, 256, 0) == 1      # one 120 x 256 tile
        assert lib.lbm_tile_count(0, 5, 0) == -1
        assert lib.lbm_tile_count(5, 5, nv) == -1
        for v in range(nv):
            tx, ty, cols = b.lbm_variant_tile(v)
            assert tx == 30 * cols and cols in (2, 4) and ty % 8 == 0
            assert b.lbm_tile_count(tx, ty, v) == 1
            assert b.lbm_tile_count(tx + 1, ty + 1, v) == 4
        with pytest.raises(b.LbmError):
            b.lbm_variant_tile(nv)
        # every variant with the clean-tile code has a twin of the same tiles
        # without it
        shapes = {v: b.lbm_variant_tile(v) for v in range(nv)}
        clean = [v for v in range(nv) if b.lbm_variant_has_clean_code(v)]
        assert clean and len(clean) < nv
        for v in clean:
            assert any(shapes[u] == shapes[v] and
                       not b.lbm_variant_has_clean_code(u) for u in range(nv))
        assert lib.lbm_variant_has_clean_code(nv) == -1
        assert lib.lbm_variant_has_clean_code(-1) == -1
    finally:
        b.lbm_destroy(ctx)
    assert b.lbm_last_error(None) == "null context"


def test_status_strings(b):
    for name in ["LBM_OK", "LBM_E_INVAL", "LBM_E_WORKSPACE", "LBM_E_CUDA",
                 "LBM_E_UNSTABLE", "LBM_E_STATE"]:
        assert b.lbm_status_string(getattr(b, name)) == name
    assert b.lbm_status_string(-99) == "LBM_E_UNKNOWN"


def test_batch_arguments_checked_on_host(b):
    lib = b._lib
    assert b.lbm_batch_workspace_bytes(0, 10) == 0
    assert b.lbm_batch_workspace_bytes(4, 0) == 0
    need = b.lbm_batch_workspace_bytes(4, 100)
    assert need > 0
    out = ctypes.c_void_p()
    assert lib.lbm_batch_create(4, 100, ctypes.c_void_p(4096 + 8), need, None,
                                ctypes.byref(out)) == b.LBM_E_WORKSPACE
    bt = b.lbm_batch_create(4, 100, 1 << 20, need)
    try:
        assert b.lbm_batch_members(bt) == 0
        assert lib.lbm_batch_add(bt, None, None) == b.LBM_E_INVAL
        p = b.make_params(20, 10)
        ctx = b.lbm_create(p, 1 << 21, b.lbm_workspace_bytes(p))
        # no geometry yet (and a different stream would also be refused)
        assert lib.lbm_batch_add(bt, ctx, None) == b.LBM_E_STATE
        b.lbm_destroy(ctx)
        assert lib.lbm_batch_remove(bt, 0) == b.LBM_E_INVAL
        assert lib.lbm_batch_set_variant(bt, b.lbm_variant_count()) == b.LBM_E_INVAL
        assert lib.lbm_batch_step(bt, -1) == b.LBM_E_INVAL
        assert lib.lbm_batch_step(bt, 3) == b.LBM_OK  # no members: no work
        assert lib.lbm_batch_autotune(bt, 3, None, None) == b.LBM_E_INVAL
    finally:
        b.lbm_batch_destroy(bt)
