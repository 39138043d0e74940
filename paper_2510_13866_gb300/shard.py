"""Chain sharding over ranks, one process per GPU.

Chains are independent Markov chains, so a multi-GPU run gives every rank its own block
of chains (disjoint Philox seeds) and runs no collective on the data path.  The only
exchange is at read-out: per-chain observables are gathered so that every rank can form
the across-chain mean and standard error over the whole job."""
import numpy as np

OBS_FIELDS = ("density", "double_occ", "m2", "ekin", "s_pipi")


def chain_seeds(rank, chains_per_rank, base=0):
    """Seeds of rank `rank`'s chains: base + rank*chains_per_rank + c, c < chains_per_rank."""
    return [int(base + rank * chains_per_rank + c) for c in range(chains_per_rank)]


def summarize(values):
    """Mean and standard error over chains of an [n_chains, n_fields] array."""
    v = np.asarray(values, dtype=np.float64)
    n = v.shape[0]
    mean = v.mean(axis=0)
    err = v.std(axis=0, ddof=1) / np.sqrt(n) if n > 1 else np.full(v.shape[1], np.nan)
    return {f: (float(m), float(e)) for f, m, e in zip(OBS_FIELDS, mean, err)}


def gather_observables(obs, device="cpu"):
    """All-gather the per-chain observables of every rank (list of dicts from
    Lattice.measure) and summarise them; every rank gets the same result.  Each rank must
    hold the same number of chains.  Without an initialised process group this is the
    local summary."""
    import torch
    import torch.distributed as dist

    local = torch.tensor([[o[f] for f in OBS_FIELDS] for o in obs], dtype=torch.float64, device=device)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return summarize(local.cpu().numpy())
    parts = [torch.empty_like(local) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, local)
    return summarize(torch.cat(parts).cpu().numpy())
