"""Chains as replicas across GPUs: chain offsets and the end-of-run reduction.

Independent Markov chains need no exchange while they sweep; each rank runs its
own chains (Philox chain index = rank * chains_per_rank + c).  The only
cross-rank step is the reduction of the per-chain accumulators
(sum s*E, sum s*docc, sum s, number of records, sum s*S_AFM) into sign-reweighted estimates
<sO>/<s> with a jackknife over chains, done by gathering the per-chain sums.
"""
import numpy as np

FIELDS = ("sE", "sD", "s", "n", "sS")
RECORD = 6          # columns of a measurement record (sign, E, docc, kinetic, running sign, S_AFM)


def chain_offset(rank, chains_per_rank):
    return rank * chains_per_rank


def chain_sums(records):
    """Per-chain sums from the per-sweep records of each chain.

    records: iterable of (n_c, RECORD) arrays (sign, E/site, docc/site, ...).
    Returns an (n_chains, 5) array of (sum s E, sum s docc, sum s, n, sum s S_AFM).
    """
    out = []
    for r in records:
        r = np.asarray(r, dtype=np.float64).reshape(-1, RECORD)
        s = r[:, 0]
        out.append([np.sum(s * r[:, 1]), np.sum(s * r[:, 2]), np.sum(s), float(len(r)),
                    np.sum(s * r[:, 5])])
    return np.array(out, dtype=np.float64).reshape(-1, len(FIELDS))


def _jackknife_ratio(num, den):
    tot_n, tot_d = num.sum(), den.sum()
    mean = tot_n / tot_d
    k = len(num)
    if k < 2:
        return float(mean), float("nan")
    jk = (tot_n - num) / (tot_d - den)
    return float(mean), float(np.sqrt((k - 1) / k * np.sum((jk - jk.mean()) ** 2)))


def pooled_estimate(sums):
    """Sign-reweighted E, docc, S_AFM and average sign with jackknife errors over chains."""
    sums = np.asarray(sums, dtype=np.float64).reshape(-1, len(FIELDS))
    E, dE = _jackknife_ratio(sums[:, 0], sums[:, 2])
    D, dD = _jackknife_ratio(sums[:, 1], sums[:, 2])
    A, dA = _jackknife_ratio(sums[:, 4], sums[:, 2])
    S, dS = _jackknife_ratio(sums[:, 2], sums[:, 3])
    return {"E": E, "E_err": dE, "docc": D, "docc_err": dD, "s_afm": A, "s_afm_err": dA,
            "sign": S, "sign_err": dS, "n_chains": int(len(sums)), "n_meas": int(sums[:, 3].sum())}


def gather_sums(local_sums, group=None):
    """All-gather the per-chain sums of every rank (torch.distributed, any
    backend); every rank gets the concatenation in rank order."""
    import torch
    import torch.distributed as dist
    nf = len(FIELDS)
    local = torch.as_tensor(np.asarray(local_sums, dtype=np.float64).reshape(-1, nf))
    world = dist.get_world_size(group)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([local.shape[0]], dtype=torch.int64), group=group)
    width = int(max(c.item() for c in counts))
    padded = torch.zeros(width, nf, dtype=torch.float64)
    padded[: local.shape[0]] = local
    parts = [torch.zeros(width, nf, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return np.concatenate([p[: int(c.item())].numpy() for p, c in zip(parts, counts)], axis=0)
