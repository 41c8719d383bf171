"""GPU parity at the full sizes of the benchmarked workloads, in the launch
configuration the benchmark times (the fused step: one graph of MD and cell
pass per interval): every particle against the FP64 oracle after one step.

- reactive sphere dimer in a 32^3 box at density 10 (327,680 solvent);
- Poiseuille channel 128^3 between stick walls at density 10 (20,971,520
  solvent, virtual wall particles, body force);
- the thermal-gradient suspension 256x64x64 (10,485,760 solvent, 64 WCA
  spheres with colloid-colloid LJ, two MPC-AT slabs), and its six-sphere
  48x32x32 version.

The comparison is the one of the reduced-size tests (keys, permutation and
flags bit-exact on the FP64 path; the mixed path within 1e-5 with key
mismatches only at cell planes, at most 1e-4 of the particles)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1608_04904_gb300 import api, build, synth
from parity_util import by_id, check_mixed_exceptions, compare_step, near_boundary, pos_bad, pos_diff, vel_bad

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


def _compare_many(cfg, st, o, precision, n_col):
    """compare_step for many colloids: on the mixed path each colloid can
    have a particle grazing its cut-off take the other branch in FP32, so the
    counts allowed grow with the number of colloids."""
    if precision == "fp64":
        compare_step(cfg, st, o, precision)
        return
    gid, gx, gv, gf, gc = by_id(st["id"], st["id"], st["x"], st["v"], st["flags"], st["cell"])
    oid, ox, ov, of, oc, onear = by_id(o.id, o.id, o.x, o.v, o.flags, o.key, o.near.astype(bool))
    assert np.array_equal(gid, oid)
    mism = gc != oc
    assert np.all(near_boundary(ox, o.shift, 1e-4)[mism]), "key mismatch away from a cell boundary"
    assert mism.sum() <= max(3, 1e-4 * len(gc))
    badcells = np.isin(oc, oc[mism]) | np.isin(oc, gc[mism])
    allow = 2 + 2 * n_col
    fd = gf != of
    check_mixed_exceptions(pos_bad(gx, ox, cfg["L"], cfg.get("walls", 0), "mixed"), onear, fd, pos_diff(gx, ox, cfg["L"], cfg.get("walls", 0)), cfg["kT"],
                           allow, "position")
    check_mixed_exceptions(vel_bad(gv, ov, cfg["kT"], "mixed") & ~badcells, onear, fd, gv - ov, cfg["kT"], allow)
    assert (gf != of).sum() <= allow + mism.sum()


@pytest.mark.parametrize("precision,size", [("fp64", "six_spheres"), ("mixed", "six_spheres"), ("mixed", "full")])
def test_thermal_suspension_step(precision, size):
    """Spheres with colloid-colloid LJ and MPC-AT slabs (the general FP64 MD
    kernel, the wide mixed one) against the oracle after one fused step."""
    if size == "full":
        cfg, col, bonds = synth.thermal(precision=precision)
    else:
        cfg, col, bonds = synth.thermal(precision=precision, L=(48, 32, 32), n_spheres=6)
    x, v, fl = synth.solvent(cfg, col, seed=cfg["seed"] + 100)
    st, cols, o = _run(cfg, col, bonds, x, v, fl, precision, step=3)
    _compare_many(cfg, st, o, precision, len(col))
    tol = 1e-10 if precision == "fp64" else 1e-5
    d = cols["x"] - o.X
    d -= np.asarray(cfg["L"], float) * np.round(d / np.asarray(cfg["L"], float))
    assert np.abs(d).max() < tol * max(cfg["L"])
