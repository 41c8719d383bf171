"""Long-run statistics of the GPU path against the oracle: the solvent
temperature T, the solvent self-diffusion coefficient D and the sphere
dimer's directed speed V, from replica ensembles of the reactive dimer
(§1.5; 16^3 box at density 10, the 32^3 nanomotor's parameters).

One-step parity bounds the arithmetic of one interval; this covers the drift
of the mixed FP32 path over thousands of intervals.  Each observable is a
per-replica time average; the spread over independent replicas gives its
standard error.  The pass rule: |difference| within 3 combined standard
errors and, for T and D, within 1 % of the reference (§1.2 names physical
validation of the velocity distribution and of the transport coefficients).
The directed speed is a small drift under thermal motion: its 1 % is below
the standard error that a test-sized ensemble reaches, so it is held to the
3-SE rule and its relative standard error is reported."""
import json
import os

import numpy as np
import pytest

from longrun_util import compare, mean_se, per_replica, run_gpu, run_oracle
from paper_1608_04904_gb300 import api, build

pytestmark = pytest.mark.gpu

R_GPU, K_GPU = 64, 2000     # replicas, production intervals (GPU paths)
R_ORC, K_ORC = 8, 400       # the oracle's ensemble (same first replicas)
WARM = 200                  # intervals before measuring (the motor's B cloud forms)


@pytest.fixture(scope="module")
def runs(orc):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()
    orc.set_threads(0)
    try:
        out = {"mixed": run_gpu(api, "mixed", R_GPU, WARM, K_GPU),
               "fp64": run_gpu(api, "fp64", R_GPU, WARM, K_GPU),
               "oracle": run_oracle(orc, R_ORC, WARM, K_ORC)}
    finally:
        orc.set_threads(1)
    return out


def _check(runs, a, b, k_max=None):
    """Compare sides a and b over the production intervals up to k_max."""
    recs, bad = [], []
    for name, need_rel in (("T", True), ("D", True), ("V", False)):
        ok, rec = compare(name, per_replica(runs[a][name], k_max), per_replica(runs[b][name], k_max),
                          need_rel=need_rel)
        rec["pair"] = f"{a} vs {b}"
        rec["intervals"] = k_max
        recs.append(rec)
        if not ok:
            bad.append(rec)
    d = os.environ.get("RMPCD_LONGRUN_LOG")
    if d:
        with open(d, "a") as f:
            for rec in recs:
                f.write(json.dumps(rec) + "\n")
    assert not bad, bad
    return recs


def test_ensembles_are_physical(runs):
    """Sanity of what is compared: T at kT = 1/3, D near the SRD closed form
    for M = 10, alpha = 90 deg, tau = 0.5, kT = 1/3 (0.194; colloids and the
    finite box lower it a little), and a motor that moves along its axis."""
    for side in ("mixed", "fp64", "oracle"):
        T, _ = mean_se(per_replica(runs[side]["T"]))
        D, _ = mean_se(per_replica(runs[side]["D"]))
        assert abs(T - 1.0 / 3.0) < 0.03 / 3.0, (side, T)
        assert 0.15 < D < 0.22, (side, D)
    V, se = mean_se(per_replica(runs["fp64"]["V"]))
    assert abs(V) > 3 * se, (V, se)


def test_mixed_matches_fp64_gpu(runs):
    """The whole run: the drift of FP32 over thousands of intervals."""
    _check(runs, "mixed", "fp64")


def test_fp64_gpu_matches_oracle(runs):
    """Over the oracle's intervals."""
    _check(runs, "fp64", "oracle", K_ORC)


def test_mixed_matches_oracle(runs):
    _check(runs, "mixed", "oracle", K_ORC)
