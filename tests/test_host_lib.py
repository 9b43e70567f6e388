"""CPU-only checks of libpqmc.so: it loads, exports every declared entry point,
and its host-side FP64 model set-up (own eigensolver) matches numpy and the
oracle.  No GPU compute is called."""
import os
import re

import numpy as np
import pytest

from oracle import lattice as olat, pqmc as opq, trial as otrial
from paper_2303_13403_gb300 import build, pqmc, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    if not os.path.exists(pqmc.LIB_PATH):
        build.build()
    return pqmc.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pqmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pqmc_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert {n for n, _, _ in pqmc.SIGNATURES} == set(names)


def test_init_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pqmc.PQMCError) as e:
        pqmc.Context([workloads.PLAIN_18])
    assert e.value.status == pqmc.ECUDA


def test_invalid_specs_rejected_before_device(lib):
    bad = [
        workloads.honeycomb(3, two_theta=1.0),                  # Ltau = 10: Ltau/2 = 5 not a multiple of 10
        workloads.honeycomb(3, two_theta=0.1),                  # Ltau odd
        workloads.ChainSpec(Lx=3, Ly=3, n_up=19),               # N_sigma > N
        workloads.ChainSpec(Lx=0, Ly=3),
        workloads.ChainSpec(Lx=3, Ly=3, dtau=-0.1),
        workloads.ChainSpec(Lx=3, Ly=3, g=-0.5),
        workloads.ChainSpec(Lx=3, Ly=3, U=-1.0),
        workloads.ChainSpec(Lx=3, Ly=3, two_theta=-0.2),
        workloads.ChainSpec(kind=7, Lx=3, Ly=3),                # unknown lattice kind
        workloads.honeycomb(23, two_theta=0.0),                 # 1058 sites: above the 1024-site maximum
        workloads.ChainSpec(kind=workloads.SQUARE, Lx=32, Ly=32, two_theta=0.0,
                            n_up=600, n_dn=600),                # N_sigma above 512
        workloads.ChainSpec(kind=workloads.HONEYCOMB_TV, Lx=3, Ly=3, n_dn=3),   # t-V has one species
    ]
    for s in bad:
        with pytest.raises(pqmc.PQMCError) as e:
            pqmc.Context([s])
        assert e.value.status == pqmc.EINVAL, s


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (18, 3), (50, 4), (97, 5)])
def test_host_eigensolver_matches_numpy(lib, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w, V = pqmc.host_eigh(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-11)
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
    assert np.allclose(V @ np.diag(w) @ V.T, A, atol=1e-11)


@pytest.mark.parametrize("L", [3, 6, 9])
def test_host_eigensolver_degenerate_lattice_spectrum(lib, L):
    K, _ = olat.honeycomb(L, L)
    w, V = pqmc.host_eigh(K)
    assert np.allclose(w, np.linalg.eigvalsh(K), atol=1e-11)
    assert np.allclose(V @ np.diag(w) @ V.T, K, atol=1e-11)


@pytest.mark.parametrize("spec", [
    workloads.PLAIN_18,
    workloads.GUTZ_72[8.0],
    workloads.DOPED_64[0.3],
    workloads.honeycomb(9, g=0.5, M_N=0.12, two_theta=8.0),
    workloads.ChainSpec(kind=workloads.SQUARE, Lx=2, Ly=4, tp=-0.2, n_up=3, n_dn=3, M_N=0.1),
])
def test_host_model_matches_oracle(lib, spec):
    p = opq.Params(kind=spec.kind, Lx=spec.Lx, Ly=spec.Ly, t=spec.t, tp=spec.tp, U=spec.U, dtau=spec.dtau,
                   two_theta=spec.two_theta, g=spec.g, M_N=spec.M_N, n_up=spec.n_up, n_dn=spec.n_dn,
                   n_stab=1 if spec.n_slices % 2 == 0 and spec.n_slices // 2 % 10 else 10)
    m = opq.Model(p)
    for spin, sigma in ((0, 1), (1, -1)):
        K, E, P, gap = pqmc.host_model(spec, spin)
        assert np.array_equal(K, m.K)
        assert np.allclose(E, m.expKm, atol=1e-13)
        # same occupied subspace: projectors agree
        Po = m.P[sigma]
        assert np.allclose(P @ P.T, Po @ Po.T, atol=1e-9)
        assert np.isclose(gap, m.gap[sigma], rtol=1e-8)


def test_variational_quadratic_minimum():
    """The refinement of the grid minimum recovers the stationary point of an
    exact paraboloid, and declines when the neighbourhood holds no minimum."""
    from paper_2303_13403_gb300 import variational
    gv = np.array(variational.G_VALUES)
    mv = np.array(variational.M_VALUES)
    G, M = np.meshgrid(gv, mv, indexing="ij")
    E = -0.9 + 0.3 * (G - 0.57) ** 2 + 0.1 * (G - 0.57) * (M - 0.08) + 2.0 * (M - 0.08) ** 2
    err = np.full_like(E, 1e-3)
    s = variational.summarise(gv, mv, E, err)
    assert s["grid_argmin"]["g"] == 0.6 and s["grid_argmin"]["M_N"] == 0.09
    f = s["fit_min"]
    assert abs(f["g"] - 0.57) < 1e-9 and abs(f["M_N"] - 0.08) < 1e-9 and abs(f["E"] + 0.9) < 1e-12
    assert variational.quadratic_minimum(gv, mv, -E, err, (5, 5)) is None
    specs = variational.grid_specs(3.5, 6)
    assert len(specs) == 121 and all(sp.two_theta == 0.0 and sp.n_sites == 72 for sp in specs)
    assert specs[12].g == 0.1 and specs[12].M_N == 0.03


def test_empty_batch_rejected(lib):
    with pytest.raises(pqmc.PQMCError) as e:
        pqmc.Context([])
    assert e.value.status == pqmc.EINVAL


def test_null_context_queries_return_zero(lib):
    """The size and count queries accept a NULL context (no device work)."""
    assert lib.pqmc_device_bytes(None) == 0
    assert lib.pqmc_upload_bytes(None) == 0
    assert lib.pqmc_num_chains(None) == -1


def test_autotune_cache_file_is_read(tmp_path):
    """The autotuner's JSON cache (PQMC_AUTOTUNE_CACHE): a stored pick for the
    batch's key is returned without timing anything (so no GPU is needed)."""
    import json
    import subprocess
    import sys
    cache = tmp_path / "tune.json"
    key = "prec1/nstab2/k0/cta0/dense0/72.36.36.40.hx4"
    cache.write_text(json.dumps({key: {"delay_k": 16, "cta_threads": 128, "ms_per_sweep": 1.5}}, indent=1))
    code = ("import json; from paper_2303_13403_gb300 import pqmc, workloads; "
            "s = workloads.honeycomb(6, two_theta=4.0, g=0.6, M_N=0.21); "
            "print(json.dumps(pqmc.autotune([s] * 4, prec=pqmc.FP32, n_stab=2)))")
    env = dict(os.environ, PQMC_AUTOTUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    t = json.loads(r.stdout.strip().splitlines()[-1])
    assert t["from_cache"] and t["delay_k"] == 16 and t["cta_threads"] == 128 and t["ms_per_sweep"] == 1.5
