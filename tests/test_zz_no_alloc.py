"""The allocation-free entry point, checked against the allocating path.

pqmc_green_noalloc serves callers that cannot allocate device memory: it puts
every buffer it needs in a fixed array inside the library and uses only the
device buffers the caller passes.  Its output (G at tau = -1 and the weight
of one chain for given fields) must equal what a context computes for the same
fields (pqmc_init_batch + pqmc_set_fields + pqmc_get_green / pqmc_get_weight),
within the FP64 parity tolerance of the other tests, on consecutive calls
that share the fixed array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2303_13403_gb300 import pqmc, workloads

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def reference(spec, fields, n_stab):
    ctx = pqmc.Context([spec], prec=pqmc.FP64, seed=1, n_stab=n_stab)
    ctx.set_fields(fields)
    G = np.stack([ctx.green(0, 0), ctx.green(0, 1)])
    w = ctx.weight()
    ctx.close()
    return G, w


@pytest.mark.parametrize("spec,n_stab", [
    (workloads.honeycomb(3, U=4.0, dtau=0.1, two_theta=2.0, g=0.6, M_N=0.21), 5),
    (workloads.GUTZ_72[4.0], 10),
])
def test_green_noalloc_matches_context(spec, n_stab):
    import torch
    torch.cuda.set_device(0)
    pqmc.load()
    N = spec.n_sites
    stream = torch.cuda.current_stream()
    for seed in (21, 22):                       # two calls in a row share the fixed array
        fields = workloads.random_fields(spec, seed)
        G_ref, w_ref = reference(spec, fields, n_stab)
        d_fields = torch.from_numpy(fields).to("cuda")
        d_G = torch.full((2, N, N), float("nan"), dtype=torch.float64, device="cuda")
        d_w = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        pqmc.green_noalloc(spec, n_stab, d_fields.data_ptr(), d_G.data_ptr(), d_w.data_ptr(), stream.cuda_stream)
        G = d_G.cpu().numpy()
        w = d_w.cpu().numpy()
        for s in (0, 1):
            assert rel_err(G[s], G_ref[s]) < 1e-10
        assert np.allclose(w[[0, 2]], w_ref[[0, 2]], rtol=1e-10, atol=1e-9)
        assert w[1] * w[3] == w_ref[1] * w_ref[3]


def test_green_noalloc_rejects_oversized_chain():
    pqmc.load()
    big = workloads.GUTZ_648            # 648 sites, 200 slices: far above the fixed array
    with pytest.raises(pqmc.PQMCError) as e:
        pqmc.green_noalloc(big, 10, 1, 1, 1)
    assert e.value.status == pqmc.EINVAL
