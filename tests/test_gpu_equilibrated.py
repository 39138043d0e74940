"""Full-size FP32 parity from equilibrated states (Sec. 3.5.2, Eq. ffbsFwd and the backward
conditional after it).

The first-sweep tests start from the static initial state, where every message is a
smooth propagator.  Here the GPU runs 100 or more sweeps first, so that the fields have
organised around the paths and the messages concentrate (kappa = max alpha / alpha(x_end)
grows); then the states of a few chains are copied into the oracle (hqmc_get_state) and
one more sweep is compared on the first 32 worldlines of each spin: the anchor, the
filter log-weights within 1e-5 relative of max(1, |log Z|) for every log-weight the
library does not flag (hqmc_logw_error), and the paths in draw order, which may differ
only at a first draw whose uniform lay within 1e-5 of a CDF edge.  The mismatch rate and
the largest log-weight error are printed.
  - L = 32, t = 1, U = 4, beta = 4, dtau = 0.05 (M = 80), half filling, 64 chains: the
    benchmark's configuration and launch;
  - L = 64, beta = 8 (M = 160), half filling, 16 chains: the large-lattice configuration.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import path_mismatches, rel_err

pytestmark = pytest.mark.gpu

NWL = 32


@pytest.mark.parametrize("L,beta,chains,sweeps,pick", [(32, 4.0, 64, 120, (0, 21, 50)),
                                                      (64, 8.0, 16, 100, (3, 12))])
def test_equilibrated_state_matches_oracle(L, beta, chains, sweeps, pick):
    from paper_2510_13866_gb300 import Lattice

    params = (1.0, 4.0, beta, 0.05, 1.0)
    lat = Lattice(L, list(range(chains)), precision="fp32")
    lat.set_params(*params)
    lat.sweep(sweeps)
    before = {c: lat.get_state(c) for c in pick}
    logw = lat.sweep(1, logw=True)
    lerr = lat.logw_error()
    nflag = sum(o["n_inexact"] for o in lat.measure(reset=True))
    draws = firsts = 0
    worst = 0.0
    for c in pick:
        s, x, _, sw = before[c]
        assert sw == sweeps
        orc = oracle.Chain(L, *params, c)
        orc.s[:] = s
        orc.x[:] = x
        orc.sweep_count = sw
        ref = orc.sweep(want_margin=True, nwl_limit=NWL)
        _, x1, a1, sw1 = lat.get_state(c)
        assert sw1 == sweeps + 1 and a1 == ref["anchor"], c
        lw, lr = logw[c][:, :NWL], ref["logw"][:, :NWL]
        err = rel_err(lw, lr)
        flagged = ~(lerr[c][:, :NWL] <= 1e-5 * np.maximum(1.0, np.abs(lw)))
        assert np.all((err <= 1e-5) | flagged), (c, err.max())
        worst = max(worst, float(err[~flagged].max()) if np.any(~flagged) else 0.0)
        d, f, bad = path_mismatches(x1, orc.x, ref["margin"], a1, orc.M, 1e-5, nwl=NWL)
        assert not bad, (c, bad[:3])
        draws += d
        firsts += f
        # the chain has left the static start: its paths move between slices
        assert np.mean(x[:, :, 1:] != x[:, :, :-1]) > 0.05
    lat.close()
    print(f"L={L}: {draws} draws compared, {firsts} first differences at CDF edges "
          f"(rate {firsts / max(1, draws):.2e}); largest unflagged log-weight error {worst:.2e}; "
          f"flagged log-weights in the last sweep: {nflag} of {chains * 2 * L * L // 2}")
