"""Checkpoint / restore on the GPU: a simulation restored from a state taken
mid-run continues bit-identically to the original (deterministic wall-hit
accumulation; 16-bit storage included, whose stochastic rounding is keyed on
the step count), in both addressings and at both step parities; rewinding a
simulation to an earlier state replays the same trajectory; a state is
refused by a simulation of another configuration."""
import numpy as np
import pytest

from tests.gpu_common import FIELDS

pytestmark = pytest.mark.gpu

BOX = dict(n=(24, 20, 40), slab=(10, 30), phi=0.62, l=3.0, seed=31, Da=1.0)
OBS = ("M_C", "M_R", "M_P", "eta", "in_C", "in_R", "out_R", "out_P", "hits_R", "hits_P", "reacted", "resid_RP")


def _sim(lbm, g, storage, layout, **kw):
    return lbm.Simulation(g, Da=BOX["Da"], n_species=2, storage=storage, layout=layout, deterministic=True, **kw)


def _snapshot(s):
    o = s.observables(profiles=False)
    return {k: s.field(k) for k in FIELDS}, {k: o[k] for k in OBS}, s.info()["step"]


def _assert_same(a, b):
    for k in FIELDS:
        np.testing.assert_array_equal(a[0][k], b[0][k], err_msg=k)
    assert a[1] == b[1]
    assert a[2] == b[2]


@pytest.mark.parametrize("storage,layout,t0", [(1, 2, 137), (0, 1, 90), (2, 2, 64)],
                         ids=["fp16-fluid-odd", "fp32-dense-even", "bf16-fluid-even"])
def test_restore_continues_bit_identically(storage, layout, t0):
    from paper_1607_02874_gb300 import lbm

    g = lbm.Geometry(*BOX["n"], slab=BOX["slab"], porosity=BOX["phi"], corr_len=BOX["l"], seed=BOX["seed"])
    a = _sim(lbm, g, storage, layout)
    a.step(t0)
    state = a.get_state()
    a.step(100)
    ref = _snapshot(a)
    assert ref[2] == t0 + 100

    b = _sim(lbm, g, storage, layout)
    b.step(3)  # its own history is overwritten by the restore
    b.set_state(state)
    assert b.info()["step"] == t0
    b.step(100)
    _assert_same(_snapshot(b), ref)

    # rewinding the original replays the same trajectory
    a.set_state(state)
    a.step(100)
    _assert_same(_snapshot(a), ref)


def test_state_of_another_configuration_is_refused():
    from paper_1607_02874_gb300 import lbm

    g = lbm.Geometry(*BOX["n"], slab=BOX["slab"], porosity=BOX["phi"], corr_len=BOX["l"], seed=BOX["seed"])
    a = _sim(lbm, g, 1, 2)
    a.step(5)
    state = a.get_state()
    for other in (_sim(lbm, g, 0, 2), _sim(lbm, g, 1, 1)):
        with pytest.raises(lbm.LbmError) as e:
            other.set_state(state)
        assert e.value.code == -1
    g2 = lbm.Geometry(*BOX["n"], slab=BOX["slab"], porosity=BOX["phi"], corr_len=BOX["l"], seed=BOX["seed"] + 1)
    with pytest.raises(lbm.LbmError):
        _sim(lbm, g2, 1, 2).set_state(state)
    with pytest.raises(lbm.LbmError):
        _sim(lbm, g, 1, 2).set_state(state[:-1])  # truncated
    bad = bytearray(state)
    bad[0] ^= 1  # magic
    with pytest.raises(lbm.LbmError):
        _sim(lbm, g, 1, 2).set_state(bytes(bad))
