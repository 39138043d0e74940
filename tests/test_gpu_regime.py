"""The paper's numerical regime (Sec. 4: t = 1, beta t = 32, dtau = 1/32 so M = 1024 slices,
FFBS blocks of 32 slices, half filling, U/t = 1 and 20), GPU against the FP64 oracle,
statistically, at L = 4 where the oracle's O(N^2) filter is cheap.

Both sides run the same Markov kernel from the same start (independent chains, disjoint
seeds), so every sweep's law is shared and the comparison does not need equilibrium.
  - Without permutations (distinguishable worldlines, sign +1): D, <m^2>, E_kin, S(pi,pi)
    and C(1,0) agree, |z| < 4.5 with the binomial two-sigma criterion.
  - With pair-swap permutation updates (Sec. 3.5.3): the mean sign agrees, and it has
    collapsed -- |<sign>| < 0.1 at beta t = 32 on both sides -- so the sign-reweighted
    fermionic observables of this regime are not reachable with this representation.
"""
import numpy as np
import pytest

import oracle
from test_gpu_accuracy import check_two_sigma, mean_se

pytestmark = pytest.mark.gpu

NAMES = ("double_occ", "m2", "ekin", "s_pipi", "c_10")
L, B = 4, 32


def gpu_rows(U, seeds, burn, meas, perm):
    from paper_2510_13866_gb300 import Lattice

    lat = Lattice(L, list(seeds), precision="fp32")
    lat.set_params(1.0, U, 32.0, 1.0 / 32.0, 1.0)
    lat.set_block(B)
    if perm:
        lat.set_permutations(True)
    lat.sweep(burn)
    lat.measure(reset=True)
    lat.sweep(meas)
    obs = lat.measure()
    lat.close()
    sg = np.array([o["mean_sign"] for o in obs])
    rows = np.array([[o["double_occ"], o["m2"], o["ekin"], o["s_pipi"], o["Cr"][1]] for o in obs])
    return rows, sg


def oracle_rows(U, seeds, burn, meas, perm):
    N = L * L
    kpp = L // 2 + L * (L // 2)
    rows, sgs = [], []
    for sd in seeds:
        ch = oracle.Chain(L, 1.0, U, 32.0, 1.0 / 32.0, 1.0, sd)
        step = (lambda: ch.perm_sweep(block=B)) if perm else (lambda: ch.sweep(block=B))
        for _ in range(burn):
            step()
        acc, sg = np.zeros(5), 0.0
        for _ in range(meas):
            r = step()
            s = r.get("sign", 1)
            m = oracle.measure(L, ch.M, r["hist"])
            MN = ch.M * N
            acc += s * np.array([m["d"] / MN, m["m2"] / MN, -(1.0 / 32.0) * r["links"].sum() / N,
                                 m["Sk"][kpp] / (4 * ch.M), m["Cr"][1] / (4 * ch.M)])
            sg += s
        rows.append(acc / meas)
        sgs.append(sg / meas)
    return np.array(rows), np.array(sgs)


@pytest.mark.parametrize("U", [1.0, 20.0])
def test_paper_regime_gpu_and_oracle_agree(U):
    burn, meas = 40, 120
    g, gs = gpu_rows(U, range(300_000, 300_256), burn, meas, perm=False)
    o, os_ = oracle_rows(U, range(310_000, 310_016), burn, meas, perm=False)
    assert np.all(gs == 1.0) and np.all(os_ == 1.0)
    (mg, sg), (mo, so) = mean_se(g), mean_se(o)
    z = (mg - mo) / np.hypot(sg, so)
    print(f"\nU={U:g}, L={L}, beta=32, M=1024, B={B}: GPU 256 chains, oracle 16, {burn}+{meas} sweeps")
    for j, n in enumerate(NAMES):
        print(f"{n:>11}: GPU {mg[j]:.6f} +- {sg[j]:.1e}  oracle {mo[j]:.6f} +- {so[j]:.1e}  z {z[j]:+.2f}")
    assert np.all(np.abs(z) < 4.5), z
    check_two_sigma(z)


@pytest.mark.parametrize("U", [1.0, 20.0])
def test_paper_regime_sign_collapses_on_both_sides(U):
    burn, meas = 40, 120
    _, gs = gpu_rows(U, range(320_000, 320_256), burn, meas, perm=True)
    _, os_ = oracle_rows(U, range(330_000, 330_016), burn, meas, perm=True)
    mg, sg = gs.mean(), gs.std(ddof=1) / np.sqrt(len(gs))
    mo, so = os_.mean(), os_.std(ddof=1) / np.sqrt(len(os_))
    z = (mg - mo) / np.hypot(sg, so)
    print(f"\nU={U:g}, permutation updates: mean sign GPU {mg:+.4f} +- {sg:.4f}, oracle {mo:+.4f} +- {so:.4f}, z {z:+.2f}")
    assert abs(z) < 4.5
    assert abs(mg) < 0.1 and abs(mg) < 0.1 + 4.5 * sg
