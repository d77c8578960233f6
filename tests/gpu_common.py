"""Helpers for the GPU parity tests: run the CUDA path (through the C ABI)
and the oracle on the same seeded inputs and compare."""
from __future__ import annotations

import numpy as np

# Field error metric: max |a - b| / max |b| over interior fluid cells, per
# field; the carrier enters as its density deviation rho_C - 1.
FIELDS = ("drho_C", "ux", "uy", "uz", "rho_R", "rho_P")


def gpu_case(case, *, n_species, steps, storage=0, layout=1, Da=1.0, p=None, pS_R=0.95, pS_P=0.0, tau=0.8,
             rho_in=1.001, rho_out=1.0, c_in=1.0, bc=0, mask=None):
    from paper_1607_02874_gb300 import lbm

    g = lbm.Geometry(case["nx"], case["ny"], case["nz"], slab=case["slab"], porosity=case["porosity"],
                     corr_len=case["corr_len"], seed=case["seed"], bc=bc, mask=mask)
    s = lbm.Simulation(g, tau=tau, rho_in=rho_in, rho_out=rho_out, c_in=c_in, Da=Da, p=p, pS_R=pS_R, pS_P=pS_P,
                       n_species=n_species, storage=storage, layout=layout)
    s.step(steps)
    out = {k: s.field(k).astype(np.float64) for k in ("drho_C", "ux", "uy", "uz", "rho_R")}
    out["rho_P"] = s.field("rho_P").astype(np.float64) if n_species == 2 else np.zeros(g.n)
    out["obs"] = s.observables()
    out["info"] = s.info()
    out["geom"] = g.info()
    out["sim"] = s
    out["g"] = g
    return out


def oracle_case(orc, case, mask, *, n_species, steps, p, pS_R=0.95, pS_P=0.0, tau=0.8, rho_in=1.001, rho_out=1.0,
                c_in=1.0, bc=0, quant=0):
    sim = orc.Sim(case["nx"], case["ny"], case["nz"], mask, n_species=n_species, tau=tau, rho_in=rho_in,
                  rho_out=rho_out, c_in=c_in, p=p, pS_R=pS_R, pS_P=pS_P, bc=bc, quant=quant)
    sim.step(steps)
    fl = sim.fields()
    ns = 1 + n_species
    out = {"drho_C": fl[0] - 1.0, "rho_R": fl[1], "rho_P": fl[2] if ns > 2 else np.zeros(sim.n),
           "ux": fl[ns], "uy": fl[ns + 1], "uz": fl[ns + 2]}
    out["obs"] = sim.observables()
    out["sim"] = sim
    return out


def interior(case, mask, bc=0):
    nz, plane = case["nz"], case["nx"] * case["ny"]
    m = mask.reshape(-1) == 0
    if bc == 0:
        z = np.arange(case["nx"] * case["ny"] * nz) // plane
        m &= (z > 0) & (z < nz - 1)
    return m


def field_errors(a, b, sel):
    errs = {}
    for k in FIELDS:
        ref = b[k][sel]
        den = np.abs(ref).max()
        if den == 0.0:
            errs[k] = float(np.abs(a[k][sel]).max())
        else:
            errs[k] = float(np.abs(a[k][sel] - ref).max() / den)
    return errs
