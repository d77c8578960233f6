"""The parameter studies, run short on the GPU so that their code paths stay
exercised: each returns its report with finite values, and the quantities
that must hold at any length hold (mass budgets close, the sweep covers its
grid, the fields of Fig. 3 are written).
"""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_precision_short():
    from paper_1607_02874_gb300 import studies

    r = studies.precision(steps=40)
    assert set(r["results"]) == {"fp32", "fp16", "bf16"}
    assert r["results"]["fp32"]["speedup_vs_fp32"] == 1.0
    for st, v in r["results"].items():
        assert v["MLUPS"] > 0 and all(math.isfinite(e) for e in v["field_err_vs_fp32"].values()), st


def test_da_sweep_short():
    from paper_1607_02874_gb300 import studies

    r = studies.da_sweep(cap=400, check=200, das=(0.1, 10.0), layouts=("fluid",))
    assert len(r["runs"]) == 2
    for run in r["runs"]:
        assert run["steps"] <= 400 and 0 < run["p"] <= 1 and math.isfinite(run["conversion_X"])
    # a smaller Da is a faster reaction: a larger p (the reactant has not
    # reached the slab in 400 steps, so the conversion is still ~0)
    assert r["runs"][0]["p"] > r["runs"][1]["p"]


def test_replica_short(tmp_path):
    from paper_1607_02874_gb300 import studies

    R = workloads.REPLICA
    r = studies.replica(steps=300)
    n = len(R["w_list"]) * len(R["p_list"]) + len(R["p_list"]) + len(R["h_list"]) - 1
    assert r["sims"] == n == len(r["runs"])
    for run in r["runs"]:
        assert abs(run["porosity"] - R["porosity"]) <= 0.005 + 1e-9  # the report rounds to 4 digits
        assert math.isfinite(run["eta"]) and math.isfinite(run["phiP_z150"])
    assert r["dimensionless"]["Kn"] == pytest.approx(0.6736, abs=1e-3)
    f = studies.replica_fig3(steps=200, save=str(tmp_path / "fig3.npz"))
    # layers from the face meeting the flow: the w = 10 ingot's ten, or the
    # first twelve of the parallel one's 200
    for orient, layers in (("perpendicular", 10), ("parallel", 12)):
        assert len(f["runs"][orient]["rhoR_by_layer_from_upstream_face"]) == layers
    arrays = np.load(tmp_path / "fig3.npz")
    assert arrays["perpendicular_rho_R"].shape == (R["nz"], R["nx"])


def test_leveque_short():
    from paper_1607_02874_gb300 import studies

    r = studies.leveque(steps=500)
    c = workloads.LEVEQUE
    assert len(r["G"]) == len(r["G_leveque"]) == c["L"]
    assert math.isfinite(r["mae_window"]) and r["u_max"] > 0


def test_serving_short():
    """The serving study on the first 6 requests with a 300-step cap: every
    request ends (capped or converged) in both storages, eta is finite and
    at least rounding-level zero (little product reaches the outlet in 300
    steps), and the FP16/FP32 comparison is reported."""
    from paper_1607_02874_gb300 import studies

    r = studies.serving(cap=300, n_requests=6, check=100)
    for name in ("fp16", "fp32"):
        s = r[name]
        assert s["status"]["converged"] + s["status"]["capped"] == 6, s["status"]
        assert s["p99_s"] >= s["p50_s"] > 0
        assert s["max_batch"] >= 1 and len(s["eta"]) == 6
        assert all(math.isfinite(v) and v > -1e-6 for v in s["eta"].values())
    assert "eta_rel_fp16_vs_fp32" in r
