"""GPU parity at the full sizes of the benchmarked workloads, in the launch
configuration the benchmark times (the fused step: one graph of MD and cell
pass per interval): every particle against the FP64 oracle after one step.

- reactive sphere dimer in a 32^3 box at density 10 (327,680 solvent);
- Poiseuille channel 128^3 between stick walls at density 10 (20,971,520
  solvent, virtual wall particles, body force).

The comparison is the one of the reduced-size tests (keys, permutation and
flags bit-exact on the FP64 path; the mixed path within 1e-5 with key
mismatches only at cell planes, at most 1e-4 of the particles).  The module
sorts last so that its long runs come after every other GPU test."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1608_04904_gb300 import api, build, synth
from parity_util import compare_step

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()


def _run(cfg, col, bonds, x, v, fl, precision, step):
    g = api.System.single(cfg, len(x), col, bonds, precision=precision, bucket_cap=64)
    g.set_state(0, x, v, fl)
    g.set_step(step)
    g.step(1)
    st = g.get_state()
    cols = g.get_colloids(0) if col else None
    g.close()
    o = orc.OracleSystem(cfg, x, v, fl, colloids=synth.colloid_arrays(col) if col else None, bonds=list(bonds),
                         step=step)
    o.step(1)
    return st, cols, o


@pytest.mark.parametrize("precision", PRECS)
def test_dimer32_full_size_step(precision):
    cfg, col, bonds = synth.dimer32(precision=precision)
    cfg["bulk_rate"] = 0.05
    x, v, fl = synth.solvent(cfg, col, seed=cfg["seed"] + 100, frac_b=0.2)
    assert len(x) == 327680
    st, cols, o = _run(cfg, col, bonds, x, v, fl, precision, step=7)
    compare_step(cfg, st, o, precision)
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert np.allclose(cols["x"], o.X, rtol=0, atol=tol * cfg["L"][0])


@pytest.mark.parametrize("precision", PRECS)
def test_poiseuille128_full_size_step(precision):
    cfg, col, bonds = synth.poiseuille(precision=precision)
    x, v, fl = synth.solvent(cfg, col, seed=cfg["seed"] + 100)
    assert len(x) == 20971520
    st, _, o = _run(cfg, col, bonds, x, v, fl, precision, step=11)
    compare_step(cfg, st, o, precision)
    # the walls hold every particle
    assert st["x"][:, 2].min() >= 0.0 and st["x"][:, 2].max() <= cfg["L"][2]
