"""The run log (pqmc_write_run_log): one JSON line per chain whose numbers
equal what pqmc_measure and the other hooks return for that chain (GPU)."""
import json

import numpy as np
import pytest

from paper_2303_13403_gb300 import pqmc, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    torch.cuda.set_device(0)
    pqmc.load()


def test_run_log_lines_match_measure(tmp_path):
    spec = workloads.honeycomb(6, U=4.0, dtau=0.1, two_theta=2.0, g=0.6, M_N=0.21)
    ctx = pqmc.Context([spec] * 4, prec=pqmc.FP32, seed=3, n_stab=2)
    ctx.sweep(2, measure=False)
    ctx.sweep(4)
    path = tmp_path / "run.jsonl"
    ctx.write_run_log(path)
    ctx.write_run_log(path)                       # appends
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 8
    for c, line in enumerate(lines[:4]):
        obs = ctx.measure(c)
        assert line["chain"] == c and line["sites"] == 72 and line["precision"] == "fp32"
        assert line["sweeps"] == 6 and line["records"] == 4
        assert line["E_per_site"] == pytest.approx(obs["E"], abs=1e-12)
        assert line["docc"] == pytest.approx(obs["docc"], abs=1e-12)
        assert line["accept"] == pytest.approx(obs["accept"], abs=1e-12)
        assert line["max_dG"] == obs["max_dG"]
        w = ctx.weight(c)
        assert line["logw"] == [w[0], w[2]]
        errs = ctx.stab_errors(c)
        assert line["stabilisations"] == len(errs) and line["dG_last"] == errs[-1]
        assert line["error"] == 0
    assert lines[4:] == lines[:4]
    ctx.close()
