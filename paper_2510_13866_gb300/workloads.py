"""Seeded synthetic workloads of the benchmark family (inputs only: lattice sizes and
model parameters per chain; none of the sampler's arithmetic).

Ragged batch: chain c draws one Philox4x64-10 block with key (1, 0) and counter
(c, 0, 0, 0) (numpy's implementation) and takes L = Ls[w0 mod 6], beta = betas[w1 mod 3],
U = Us[w2 mod 3], filling = fills[w3 mod 3]; its own seed is c.  t = 1, dtau = 0.05.
"""
import numpy as np

RAGGED_L = (8, 12, 16, 24, 32, 48)
RAGGED_BETA = (2.0, 4.0, 6.0)
RAGGED_U = (2.0, 4.0, 8.0)
RAGGED_FILL = (0.5, 0.875, 1.0)


def philox_block(counter, key):
    """Four 64-bit words of Philox4x64-10 at the 256-bit counter `counter` (an int)."""
    bg = np.random.Philox(counter=(int(counter) - 1) % 2**256, key=int(key))
    return [int(w) for w in bg.random_raw(4)]


def ragged(n_chains=256, t=1.0, dtau=0.05):
    """[(L, (t, U, beta, dtau, filling), seed)] for chains c = 0..n_chains-1."""
    out = []
    for c in range(n_chains):
        w = philox_block(c, 1)
        L = RAGGED_L[w[0] % 6]
        params = (t, RAGGED_U[w[2] % 3], RAGGED_BETA[w[1] % 3], dtau, RAGGED_FILL[w[3] % 3])
        out.append((L, params, c))
    return out
