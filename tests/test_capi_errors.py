"""Argument errors of the C ABI, checked without a GPU: every entry point
validates its arguments before any CUDA call and answers LBM_ERR_ARG with a
message in lbm_last_error; the error strings cover every status code; the
request footprint (host arithmetic only) orders storages and sizes."""
import ctypes

import pytest

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_DIVERGED, LBM_ERR_STATE, LBM_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6


@pytest.fixture(scope="module")
def lib():
    from paper_1607_02874_gb300 import build, lbm

    build.build()
    return lbm.library()


def _desc(lbm, **kw):
    d = dict(nx=8, ny=8, nz=16, slab_z0=4, slab_z1=12, porosity=0.6, corr_len=2.0, seed=1, mask=None,
             bc_z=lbm.BC_PRESSURE)
    d.update(kw)
    return lbm.lbm_geometry_desc(*d.values())


def _params(lbm, **kw):
    p = dict(tau=0.8, rho_in=1.001, rho_out=1.0, c_in=1.0, Da=1.0, p_override=-1.0, pS_R=0.95, pS_P=0.0,
             n_species=2, storage=lbm.FP32, layout=lbm.LAYOUT_AUTO, deterministic=0)
    p.update(kw)
    return lbm.lbm_params(**p)


def _footprint(lib, lbm, d, p):
    out = ctypes.c_size_t()
    rc = lib.lbm_request_footprint(ctypes.byref(d), ctypes.byref(p), ctypes.byref(out))
    return rc, out.value


def test_error_strings_cover_every_code(lib):
    seen = set()
    for code in (LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_DIVERGED, LBM_ERR_STATE, LBM_ERR_TIMEOUT):
        s = lib.lbm_error_string(code)
        assert s and s not in seen, code
        seen.add(s)
    assert b"diverged" in lib.lbm_error_string(LBM_ERR_DIVERGED)
    assert lib.lbm_error_string(-99)  # unknown codes still give a string


@pytest.mark.parametrize("kw,msg", [
    (dict(nz=3), b"at least"),
    (dict(nx=0), b"at least"),
    (dict(bc_z=7), b"bc_z"),
    (dict(slab_z0=10, slab_z1=4), b"slab"),
    (dict(slab_z1=17), b"slab"),
    (dict(porosity=1.5), b"porosity"),
    (dict(porosity=float("nan")), b"porosity"),
    (dict(corr_len=-1.0), b"corr_len"),
])
def test_create_geometry_rejects_bad_descriptions(lib, kw, msg):
    from paper_1607_02874_gb300 import lbm

    d = _desc(lbm, **kw)
    h = ctypes.c_void_p(1234)
    assert lib.lbm_create_geometry(ctypes.byref(d), None, None, ctypes.byref(h)) == LBM_ERR_ARG
    assert msg in lib.lbm_last_error()


def test_create_geometry_rejects_unknown_mask_values(lib):
    from paper_1607_02874_gb300 import lbm

    import numpy as np

    m = np.zeros(8 * 8 * 16, np.uint8)
    m[6 * 64 + 10] = 3  # 0 fluid, 1 catalytic, 2 inert: nothing else
    d = _desc(lbm, mask=m.ctypes.data_as(ctypes.c_void_p))
    h = ctypes.c_void_p()
    assert lib.lbm_create_geometry(ctypes.byref(d), None, None, ctypes.byref(h)) == LBM_ERR_ARG
    assert b"mask values" in lib.lbm_last_error()


def test_create_geometry_rejects_solid_next_to_inlet(lib):
    from paper_1607_02874_gb300 import lbm

    import numpy as np

    m = np.zeros(8 * 8 * 16, np.uint8)
    m[1 * 64 + 10] = 1  # a solid cell in plane 1, next to the inlet plane
    d = _desc(lbm, mask=m.ctypes.data_as(ctypes.c_void_p))
    h = ctypes.c_void_p()
    assert lib.lbm_create_geometry(ctypes.byref(d), None, None, ctypes.byref(h)) == LBM_ERR_ARG
    assert b"inlet/outlet" in lib.lbm_last_error()


@pytest.mark.parametrize("kw,msg", [
    (dict(tau=0.5), b"tau"),
    (dict(tau=float("nan")), b"tau"),
    (dict(n_species=3), b"n_species"),
    (dict(storage=9), b"storage"),
    (dict(layout=5), b"layout"),
    (dict(pS_R=1.5), b"sticking"),
    (dict(pS_P=-0.1), b"sticking"),
    (dict(rho_in=0.0), b"densities"),
    (dict(c_in=-1.0), b"densities"),
    (dict(sputter=5), b"sputter"),
    (dict(velocity=3), b"velocity"),
    (dict(inlet=4), b"inlet"),
    (dict(inlet=1, u_in=0.5), b"u_in"),
    (dict(inlet=1, u_in=float("nan")), b"u_in"),
    (dict(tau_s=0.5), b"tau_s"),
    (dict(g_z=0.02), b"g_z"),
    (dict(g_z=float("nan")), b"g_z"),
    (dict(g_z=1e-5, velocity=1), b"body force"),
    (dict(g_z=1e-5, storage=1), b"FP32"),
    (dict(desorb=2), b"desorb"),
    (dict(sputter=2, velocity=1), b"bounce-back"),
])
def test_params_are_validated(lib, kw, msg):
    from paper_1607_02874_gb300 import lbm

    rc, _ = _footprint(lib, lbm, _desc(lbm), _params(lbm, **kw))
    assert rc == LBM_ERR_ARG
    assert msg in lib.lbm_last_error()
    # lbm_init refuses a missing geometry before any device work
    s = ctypes.c_void_p(1234)
    p = _params(lbm, **kw)
    assert lib.lbm_init(None, ctypes.byref(p), None, None, ctypes.byref(s)) == LBM_ERR_ARG


def test_footprint_orders_storage_and_size(lib):
    from paper_1607_02874_gb300 import lbm

    fp = {}
    for st in (lbm.FP32, lbm.FP16_DEV, lbm.BF16_DEV):
        rc, fp[st] = _footprint(lib, lbm, _desc(lbm, nx=64, ny=64, nz=64), _params(lbm, storage=st))
        assert rc == LBM_OK
    assert fp[lbm.FP16_DEV] == fp[lbm.BF16_DEV] < fp[lbm.FP32]
    # the populations dominate: at least 3 arrays x 19 x 2 bytes per cell
    assert fp[lbm.FP16_DEV] >= 64 ** 3 * 3 * 19 * 2
    rc, big = _footprint(lib, lbm, _desc(lbm, nx=64, ny=64, nz=128), _params(lbm))
    assert rc == LBM_OK and big > 1.9 * fp[lbm.FP32]
    rc, one = _footprint(lib, lbm, _desc(lbm, nx=64, ny=64, nz=64), _params(lbm, n_species=1))
    assert rc == LBM_OK and one < fp[lbm.FP32]
    # the random sputtering matrix keeps one accumulator per (node, link)
    rc, rnd = _footprint(lib, lbm, _desc(lbm, nx=64, ny=64, nz=64), _params(lbm, sputter=lbm.SPUTTER_RANDOM))
    assert rc == LBM_OK and rnd > fp[lbm.FP32]


def test_null_handles_are_argument_errors(lib):
    from paper_1607_02874_gb300 import lbm

    n = ctypes.c_size_t()
    o = lbm.lbm_obs()
    assert lib.lbm_step(None, 1) == LBM_ERR_ARG
    assert lib.lbm_step_batch(None, 1, 1, None) == LBM_ERR_ARG
    assert lib.lbm_observables(None, ctypes.byref(o)) == LBM_ERR_ARG
    assert lib.lbm_observables_noalloc(None, ctypes.byref(o)) == LBM_ERR_ARG
    assert lib.lbm_state_size(None, ctypes.byref(n)) == LBM_ERR_ARG
    assert lib.lbm_get_state(None, None, 0) == LBM_ERR_ARG
    assert lib.lbm_set_state(None, None, 0) == LBM_ERR_ARG
    assert lib.lbm_get_field(None, 0, None, 0) == LBM_ERR_ARG
    assert lib.lbm_geometry_info(None, None, None, None, None) == LBM_ERR_ARG
    counts = (ctypes.c_int64 * 4)()
    assert lib.lbm_warp_counts(None, counts) == LBM_ERR_ARG
    assert lib.lbm_step_timed(None, None, None) == LBM_ERR_ARG
    assert lib.lbm_sim_info(None, None, None, None, None) == LBM_ERR_ARG
    passed = ctypes.c_int()
    for args in ((0, 1, 1.0), (9, 1, 1.0), (2, 0, 1.0), (2, 65, 1.0), (2, 2, 0.0), (2, 2, 11.0)):
        assert lib.lbm_selftest_barrier(*args, None, ctypes.byref(passed)) == LBM_ERR_ARG, args
    lib.lbm_destroy(None)  # no-ops
    lib.lbm_geometry_free(None)
