"""The synthetic ragged batch (256 chains over L in {8,12,16,24,32,48}, beta in {2,4,6},
U in {2,4,8}, filling in {0.5,0.875,1}, dtau = 0.05): host logic only, no GPU."""
import math
from collections import Counter

from paper_2510_13866_gb300.workloads import RAGGED_BETA, RAGGED_FILL, RAGGED_L, RAGGED_U, ragged


def test_ragged_batch_covers_every_value_and_is_valid():
    work = ragged(256)
    assert len(work) == 256
    assert [sd for _, _, sd in work] == list(range(256))
    cnt = {k: Counter() for k in ("L", "U", "beta", "fill")}
    for L, (t, U, beta, dtau, fill), _ in work:
        assert t == 1.0 and dtau == 0.05
        cnt["L"][L] += 1
        cnt["U"][U] += 1
        cnt["beta"][beta] += 1
        cnt["fill"][fill] += 1
        # an integer number of slices and of worldlines per spin, as the library requires
        M = beta / dtau
        assert abs(M - round(M)) < 1e-9 and round(M) in (40, 80, 120)
        nsig = fill * L * L / 2
        assert abs(nsig - round(nsig)) < 1e-9 and 1 <= round(nsig) <= L * L
    assert set(cnt["L"]) == set(RAGGED_L) and set(cnt["U"]) == set(RAGGED_U)
    assert set(cnt["beta"]) == set(RAGGED_BETA) and set(cnt["fill"]) == set(RAGGED_FILL)
    # each value of a uniform draw over k options: about 256/k chains (4 sigma band)
    for key, k in (("L", 6), ("U", 3), ("beta", 3), ("fill", 3)):
        mean = 256 / k
        sd = math.sqrt(256 * (1 / k) * (1 - 1 / k))
        assert all(abs(n - mean) < 4 * sd for n in cnt[key].values()), (key, cnt[key])


def test_ragged_batch_is_a_prefix_stable_function_of_the_chain_index():
    assert ragged(16) == ragged(256)[:16]
    assert ragged(8) == ragged(8)
