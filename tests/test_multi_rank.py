"""The N>1 path on CPU: two gloo ranks, each with its own chains; the gathered
per-chain sums give the same pooled estimate as one process holding all chains."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2303_13403_gb300 import distributed


def synthetic_records(chain, n=40):
    rng = np.random.default_rng(1000 + chain)
    s = np.where(rng.random(n) < 0.9, 1.0, -1.0)
    E = -0.8 + 0.05 * rng.standard_normal(n)
    D = 0.12 + 0.01 * rng.standard_normal(n)
    A = 0.03 + 0.005 * rng.standard_normal(n)
    return np.column_stack([s, E, D, E, s, A])


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, per_rank, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off = distributed.chain_offset(rank, per_rank[0])
    mine = [synthetic_records(off + c) for c in range(per_rank[rank])]
    allsums = distributed.gather_sums(distributed.chain_sums(mine))
    est = distributed.pooled_estimate(allsums)
    out.put((rank, off, est, allsums.shape))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_equals_single_process():
    per_rank = [5, 5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, per_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [0, 5]                      # distinct Philox chain indices
    ref = distributed.pooled_estimate(distributed.chain_sums([synthetic_records(c) for c in range(10)]))
    for _, _, est, shape in res:
        assert shape == (10, 5)
        for k in ("E", "E_err", "docc", "docc_err", "s_afm", "s_afm_err", "sign", "sign_err"):
            assert np.isclose(est[k], ref[k], rtol=1e-12, atol=0), k


def test_pooled_estimate_matches_direct_ratio():
    recs = [synthetic_records(c) for c in range(6)]
    est = distributed.pooled_estimate(distributed.chain_sums(recs))
    allr = np.concatenate(recs)
    assert np.isclose(est["E"], np.sum(allr[:, 0] * allr[:, 1]) / np.sum(allr[:, 0]), rtol=1e-14)
    assert np.isclose(est["sign"], np.mean(allr[:, 0]), rtol=1e-14)
    assert np.isclose(est["s_afm"], np.sum(allr[:, 0] * allr[:, 5]) / np.sum(allr[:, 0]), rtol=1e-14)
    assert est["n_meas"] == 240 and est["E_err"] > 0
