"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

  - integer geometry (mask, fluid / node numbering, b(x), link list, chord
    length) bit-exact;
  - FP32 fields within 1e-5 max relative error (carrier as rho_C - 1), both
    addressing modes, both step parities, several blocks and ragged tails;
  - observables (masses, flows, wall hits, eta, residuals) against the
    oracle's, and the FP64 plane reductions against a host FP64 sum of the
    GPU's own exported fields;
  - reduced-precision storage against the oracle run with the same storage
    rounding emulated, and against the exact oracle.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_common import field_errors, gpu_case, interior, oracle_case

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _orc_mask(orc, case, bc=0):
    return orc.geometry(case["nx"], case["ny"], case["nz"], case["slab"][0], case["slab"][1], case["porosity"],
                        case["corr_len"], case["seed"])


GEOM_CASES = [workloads.CFG1, workloads.ragged_case()]


@pytest.mark.parametrize("case", GEOM_CASES, ids=lambda c: c["name"])
@pytest.mark.parametrize("bc", [0, 1])
def test_geometry_bit_exact(orc, case, bc):
    from paper_1607_02874_gb300 import lbm

    mask = _orc_mask(orc, case)
    if bc == 0 and (mask.reshape(case["nz"], -1)[[0, 1, -2, -1]].any()):
        pytest.skip("slab touches the inlet/outlet planes")
    g = lbm.Geometry(case["nx"], case["ny"], case["nz"], slab=case["slab"], porosity=case["porosity"],
                     corr_len=case["corr_len"], seed=case["seed"], bc=bc)
    ex = g.export(links=True)
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    np.testing.assert_array_equal(ex["mask"], mask)
    fi, ni, nf, nn = orc.index_maps(nx, ny, nz, mask, zper=bool(bc))
    np.testing.assert_array_equal(ex["fluid_idx"], fi)
    np.testing.assert_array_equal(ex["node_idx"], ni)
    np.testing.assert_array_equal(ex["b"], orc.active_links(nx, ny, nz, mask, zper=bool(bc)))
    np.testing.assert_array_equal(ex["links"], orc.links(nx, ny, nz, mask, zper=bool(bc)))
    info = g.info()
    assert info["n_fluid"] == nf and info["n_nodes"] == nn
    assert info["delta"] == orc.chord_length(nx, ny, nz, case["slab"][0], case["slab"][1], mask)


def test_caller_mask_matches_generated(orc):
    from paper_1607_02874_gb300 import lbm

    case = workloads.ragged_case()
    mask = _orc_mask(orc, case)
    g = lbm.Geometry(case["nx"], case["ny"], case["nz"], slab=case["slab"], mask=mask)
    np.testing.assert_array_equal(g.export()["mask"], mask)
    assert g.info()["delta"] == orc.chord_length(case["nx"], case["ny"], case["nz"], *case["slab"], mask)


def test_inlet_plane_solid_rejected():
    from paper_1607_02874_gb300 import lbm

    mask = np.zeros((8, 6, 6), np.uint8)
    mask[1, 2, 2] = 1
    with pytest.raises(lbm.LbmError):
        lbm.Geometry(6, 6, 8, mask=mask.reshape(-1))


PARITY = [
    # (case, n_species, steps, p or None (from Da), pS_P)
    (workloads.CFG1, 1, 500, None, 0.0),
    (workloads.ragged_case(), 2, 301, 0.45, 0.1),
    (workloads.ragged_case(), 2, 120, 1.0, 0.0),
]


@pytest.mark.parametrize("layout", [1, 2], ids=["dense", "fluid"])
@pytest.mark.parametrize("pc", PARITY, ids=lambda p: f"{p[0]['name']}-S{p[1] + 1}-t{p[2]}")
def test_fp32_fields_and_observables(orc, pc, layout):
    case, nsp, steps, p, pS_P = pc
    mask = _orc_mask(orc, case)
    gp = gpu_case(case, n_species=nsp, steps=steps, layout=layout, p=p, pS_P=pS_P, Da=case.get("Da", 1.0))
    p_used = gp["info"]["p"]
    if p is None:
        assert p_used == pytest.approx(orc.reaction_probability(case["Da"], gp["geom"]["delta"]), rel=1e-15)
    oc = oracle_case(orc, case, mask, n_species=nsp, steps=steps, p=p_used, pS_P=pS_P)
    sel = interior(case, mask)
    errs = field_errors(gp, oc, sel)
    print("fp32 field errors", case["name"], layout, errs)
    for k, e in errs.items():
        assert e <= FP32_TOL, (k, e)
    go, oo = gp["obs"], oc["obs"]
    scale_R = max(abs(oo["M_R"]), 1e-30)
    # plane sums inherit the field tolerance
    for k in ("M_C", "M_R", "M_P"):
        assert abs(go[k] - oo[k]) <= FP32_TOL * max(abs(oo[k]), 1e-30) + 1e-9 * scale_R, (k, go[k], oo[k])
    for k in ("in_R", "out_R", "hits_R", "reacted", "stuck_R", "in_P", "out_P", "hits_P"):
        assert abs(go[k] - oo[k]) <= FP32_TOL * max(abs(oo[k]), abs(oo["in_R"]), 1e-30), (k, go[k], oo[k])
    for k in ("in_C", "out_C"):
        assert abs(go[k] - oo[k]) <= FP32_TOL * max(abs(oo[k]), 1e-6), (k, go[k], oo[k])
    if abs(oo["eta"]) > 1e-6:
        assert go["eta"] == pytest.approx(oo["eta"], rel=FP32_TOL)
    # the GPU's own mass budget closes (FP64 sums over an FP32 state: the
    # stored populations are rounded every step, so the budget drifts by
    # ~1e-8 of the mass per step, ~1e-5 over the 500-step case)
    assert abs(go["resid_C"]) <= 1e-5 * abs(oo["in_C"] - oo["out_C"]) + 1e-7 * go["M_C"]
    assert abs(go["resid_RP"]) <= 5e-5 * max(oo["in_R"], 1e-30)
    # per-layer profiles: densities and flux inherit the field tolerance; the
    # wall-hit profile is a sum over wall-adjacent post-collision populations
    # of one step, whose relative FP32 error is a few times the
    # max-normalised field error
    for k, tol in (("rhoR_z", FP32_TOL), ("phiP_z", FP32_TOL), ("react_z", 5 * FP32_TOL)):
        ref = oo[k]
        den = np.abs(ref).max()
        if den > 0:
            assert np.abs(go[k] - ref).max() / den <= tol, k


@pytest.mark.parametrize("layout", [1, 2], ids=["dense", "fluid"])
def test_deterministic_accumulation_matches_oracle(orc, layout):
    # the fixed-point wall-hit sums (deterministic mode) meet the same bound
    from paper_1607_02874_gb300 import lbm

    case = workloads.ragged_case()
    mask = _orc_mask(orc, case)
    g = lbm.Geometry(case["nx"], case["ny"], case["nz"], slab=case["slab"], porosity=case["porosity"],
                     corr_len=case["corr_len"], seed=case["seed"])
    s = lbm.Simulation(g, n_species=2, p=0.45, pS_P=0.1, layout=layout, deterministic=True)
    s.step(201)
    gp = {k: s.field(k).astype(np.float64) for k in ("drho_C", "ux", "uy", "uz", "rho_R", "rho_P")}
    oc = oracle_case(orc, case, mask, n_species=2, steps=201, p=0.45, pS_P=0.1)
    errs = field_errors(gp, oc, interior(case, mask))
    for k, e in errs.items():
        assert e <= FP32_TOL, (k, e)
    o = s.observables()
    assert o["hits_R"] == pytest.approx(oc["obs"]["hits_R"], rel=FP32_TOL)


def test_fp64_plane_reduction_against_host_sum(orc):
    case = workloads.ragged_case()
    gp = gpu_case(case, n_species=2, steps=40, layout=2, p=0.45)
    s = gp["sim"]
    mask = gp["g"].export()["mask"]
    nz, plane = case["nz"], case["nx"] * case["ny"]
    rR = s.field("rho_R").astype(np.float64).reshape(nz, plane)
    d = s.field("drho_C").astype(np.float64).reshape(nz, plane)
    fl = (mask.reshape(nz, plane) == 0)
    o = gp["obs"]
    for z in range(1, nz - 1):
        assert o["rhoR_z"][z] == pytest.approx(rR[z][fl[z]].sum(), rel=1e-6, abs=1e-12)
        # the export and the plane sums each form the cell's rho_C - 1 in
        # FP32 (FMA contraction may differ by an ulp of ~1e-3 per cell); an
        # FP32 plane sum would be off by ~1e-7
        assert o["rhoC_z"][z] == pytest.approx((1.0 + d[z][fl[z]]).sum(), rel=1e-10)


def test_dense_and_fluid_only_agree(orc):
    case = workloads.ragged_case()
    a = gpu_case(case, n_species=2, steps=151, layout=1, p=0.3, pS_P=0.05)
    b = gpu_case(case, n_species=2, steps=151, layout=2, p=0.3, pS_P=0.05)
    sel = interior(case, a["g"].export()["mask"])
    errs = field_errors(a, b, sel)
    for k, e in errs.items():
        assert e <= 1e-6, (k, e)


@pytest.mark.parametrize("storage,quant", [(1, 1), (2, 2)], ids=["fp16", "bf16"])
def test_reduced_precision(orc, storage, quant):
    case = workloads.ragged_case()
    mask = _orc_mask(orc, case)
    gp = gpu_case(case, n_species=2, steps=200, storage=storage, layout=2, p=0.45)
    emu = oracle_case(orc, case, mask, n_species=2, steps=200, p=0.45, quant=quant)
    exact = oracle_case(orc, case, mask, n_species=2, steps=200, p=0.45, quant=0)
    sel = interior(case, mask)
    e_emu = field_errors(gp, emu, sel)
    e_exact = field_errors(gp, exact, sel)
    e_q = field_errors(emu, exact, sel)
    print("storage", storage, "vs emulation", e_emu, "vs exact", e_exact, "emulation vs exact", e_q)
    # the GPU error against the exact oracle is the storage rounding's own
    # error (seen in the emulation) plus FP32 noise: at most twice it
    for k in e_exact:
        assert e_exact[k] <= 2.0 * e_q[k] + 1e-5, (k, e_exact[k], e_q[k])


REPORT_KEYS = ("M_C", "M_R", "M_P", "eta", "in_C", "out_C", "in_R", "out_R", "in_P", "out_P", "hits_R", "hits_P",
               "reacted", "stuck_R")


@pytest.mark.parametrize("layout", [2], ids=["fluid"])
def test_fp64_reductions_error_per_result(orc, layout):
    """Relative error of every FP64 reduction result against the FP64 oracle
    on the ragged C+R+P case (FP32 state, 301 steps), printed as a table. A
    result's scale is its own magnitude (flows and hits: at least the
    reactant inflow, whose size sets what an error in them means)."""
    case = workloads.ragged_case()
    mask = _orc_mask(orc, case)
    gp = gpu_case(case, n_species=2, steps=301, layout=layout, p=0.45, pS_P=0.1)
    oc = oracle_case(orc, case, mask, n_species=2, steps=301, p=0.45, pS_P=0.1)
    go, oo = gp["obs"], oc["obs"]
    rows = []
    for k in REPORT_KEYS:
        scale = abs(oo[k]) if k in ("M_C", "M_R", "M_P", "eta") else max(abs(oo[k]), abs(oo["in_R"]))
        if k in ("in_C", "out_C"):
            scale = max(abs(oo[k]), 1e-6)
        err = abs(go[k] - oo[k]) / scale if scale > 0 else abs(go[k])
        rows.append((k, oo[k], go[k], err))
    print("\nresult | oracle (FP64) | GPU | relative error")
    for k, o, g, e in rows:
        print(f"{k} | {o:.10g} | {g:.10g} | {e:.2e}")
    for k, o, g, e in rows:
        if k == "eta" and abs(o) < 1e-6:
            continue
        assert e <= FP32_TOL, (k, o, g, e)
