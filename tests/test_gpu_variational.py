"""The Theta = 0 variational scan (Method section, Fig. 1) on the GPU: every
(g, M_N) point of an 11 x 11 grid on the 8-site honeycomb cluster, 16 chains
per point in one context, against the exact variational energy
<psi_G|H|psi_G>/<psi_G|psi_G> from Fock space."""
import numpy as np
import pytest

from oracle import ed, pqmc as opq
from paper_2303_13403_gb300 import pqmc, variational

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    torch.cuda.set_device(0)
    pqmc.load()


def exact_grid(U, L, gv, mv, dtau=0.1):
    E = np.zeros((len(gv), len(mv)))
    cluster = None
    for i, g in enumerate(gv):
        for j, m in enumerate(mv):
            model = opq.Model(opq.Params(Lx=L, Ly=L, U=U, dtau=dtau, two_theta=0.0, g=g, M_N=m, n_stab=1))
            if cluster is None:
                cluster = ed.Cluster(model.K, model.n_sigma[1], model.n_sigma[-1], U)
            E[i, j] = cluster.trotter_projection(model.P[1], model.P[-1], g, dtau, 0)[0] / model.N
    return E


def test_variational_grid_matches_fock_space():
    U, L = 4.0, 2
    gv, mv = variational.G_VALUES, variational.M_VALUES
    r = variational.scan([U], L, chains_per_point=16, n_warm=20, n_meas=150)
    assert r["chains"] == 121 * 16
    x = r[U]
    Ex = exact_grid(U, L, gv, mv)
    # g = 0: lambda = 0, every field configuration has the same weight and the
    # same G, so the estimate is the exact Slater-state energy with no noise
    assert gv[0] == 0.0 and np.all(x["E_err"][0] < 1e-12)
    assert np.abs(x["E"][0] - Ex[0]).max() < 1e-10
    z = (x["E"][1:] - Ex[1:]) / x["E_err"][1:]
    assert np.all(np.isfinite(z))
    assert np.mean(z ** 2) < 2.0, np.mean(z ** 2)
    assert np.abs(z).max() < 6.0, np.abs(z).max()
    assert np.all(x["sign"] == 1.0)                    # Theta = 0 weights are positive
    # the grid argmin of the Monte Carlo energies is a near-optimal point of
    # the exact surface
    a = x["grid_argmin"]
    i, j = gv.index(a["g"]), mv.index(a["M_N"])
    assert Ex[i, j] - Ex.min() < 3.0 * np.median(x["E_err"])
