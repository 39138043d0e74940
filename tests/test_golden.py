"""The oracle against its stored regression fixture (tests/golden/l4_beta2_first_sweeps.json,
written by tests/golden/make_golden.py from oracle/ alone), and the FP64 GPU context
against the same fixture."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
FIX = json.load(open(os.path.join(HERE, "golden", "l4_beta2_first_sweeps.json")))


def test_oracle_reproduces_fixture(orc):
    p = FIX["params"]
    ch = orc.Chain(p["L"], p["t"], p["U"], p["beta"], p["dtau"], p["filling"], p["seed"])
    for k in range(FIX["sweeps"]):
        r = ch.sweep()
        assert r["anchor"] == FIX["anchors"][k]
        assert np.allclose(r["logw"], FIX["logw"][k], rtol=1e-13, atol=0)
    assert np.array_equal(ch.x, np.array(FIX["x"]))
    assert np.array_equal(ch.s, np.array(FIX["s"]))


@pytest.mark.gpu
def test_gpu_fp64_reproduces_fixture():
    from paper_2510_13866_gb300 import Lattice

    p = FIX["params"]
    lat = Lattice(p["L"], [p["seed"]], precision="fp64")
    lat.set_params(p["t"], p["U"], p["beta"], p["dtau"], p["filling"])
    for k in range(FIX["sweeps"]):
        lw = lat.sweep(1, logw=True)[0]
        _, _, a, _ = lat.get_state(0)
        assert a == FIX["anchors"][k]
        assert np.abs(lw - np.array(FIX["logw"][k])).max() <= 1e-12 * np.abs(lw).max()
    s, x, _, _ = lat.get_state(0)
    assert np.array_equal(x, np.array(FIX["x"]))
    assert np.array_equal(s, np.array(FIX["s"]))
    lat.close()
