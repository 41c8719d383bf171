"""GPU parity of the slab profile (rmpcd_profile, the flow / temperature /
species profiles of §"Applications of RMPCDMD"): the CUDA kernel through the C
ABI against the oracle's definition on the GPU's own stored state.  The
profile is fixed point, so counts and sums must match bit for bit; the
Poiseuille flow it measures is checked against the closed-form viscosity."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1608_04904_gb300 import api, build, synth

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()


def _expect(s, r, axis, n_bins):
    st = s.get_state(r)
    L = s.replicas[r]["cfg"]["L"][axis]
    return orc.slab_profile(L, st["x"][:, axis], st["v"], st["flags"], n_bins)


def _same(got, want):
    for k in ("n", "n_B", "v_sum", "v2_sum"):
        assert np.array_equal(got[k], want[k]), k


@pytest.mark.parametrize("precision", PRECS)
def test_profile_bit_exact_after_steps(precision):
    """Walls, body force and B species; profiles along every axis after a few
    fused steps, with one bin per cell, a ragged bin count and one bin."""
    cfg = synth.base_config(L=(20, 14, 11), walls=1, rho_wall=10, g=(0.01, 0.0, 0.0), kT=1.0, seed=21,
                            precision=precision)
    x, v, fl = synth.solvent(cfg, seed=21, frac_b=0.35)
    s = api.System([dict(cfg=cfg, n=len(x))], precision, 64)
    s.set_state(0, x, v, fl)
    s.step(4)
    for axis, n_bins in [(2, 11), (0, 7), (1, 1), (2, 512)]:
        _same(s.profile(0, axis, n_bins), _expect(s, 0, axis, n_bins))


@pytest.mark.parametrize("precision", PRECS)
def test_profile_of_each_replica_in_a_batch(precision):
    """Replicas of different sizes, one with a colloid and one with a Janus
    body: each profile sees its own replica only."""
    reps = []
    for k, side in enumerate((10, 14, 12)):
        cfg = synth.base_config(L=(side, side, side), kT=1.0, seed=30 + k, precision=precision, tau=0.5,
                                n_md=10)
        rep = dict(cfg=cfg)
        if k == 1:
            col = [dict(x=[7.0, 7.0, 7.0], v=[0.0, 0.0, 0.0], mass=500.0, sigma=2.0, eps_A=1.0, eps_B=1.0,
                        catalytic=1)]
            x, v, fl = synth.solvent(cfg, col, seed=40 + k)
            rep["colloids"] = col
        elif k == 2:
            body = synth.janus_body(60, (6.1, 5.9, 6.0), seed=k, radius=2.5)
            x, v, fl = synth.solvent(cfg, synth.body_exclusion(body), seed=40 + k)
            rep["body"] = body
        else:
            x, v, fl = synth.solvent(cfg, seed=40 + k)
        rep.update(n=len(x), state=(x, v, fl))
        reps.append(rep)
    s = api.System([{k: r[k] for k in r if k != "state"} for r in reps], precision, 64)
    for i, r in enumerate(reps):
        s.set_state(i, *r["state"])
    s.step(2)
    for i in range(3):
        got = s.profile(i, 0, 9)
        _same(got, _expect(s, i, 0, 9))
        assert got["n"].sum() == reps[i]["n"]


@pytest.mark.parametrize("precision", PRECS)
def test_profile_before_any_step_and_empty_bins(precision):
    """Straight after set_state: particles only in the lower half of the box,
    so the upper bins are empty (zero count and zero sums)."""
    cfg = synth.base_config(L=(8, 8, 8), kT=1.0, seed=5, precision=precision)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (3000, 3)) * [8.0, 8.0, 4.0]
    v = rng.normal(0, 1, (3000, 3))
    s = api.System([dict(cfg=cfg, n=len(x))], precision, 64)
    s.set_state(0, x, v, None)
    got = s.profile(0, 2, 16)
    _same(got, _expect(s, 0, 2, 16))
    assert np.all(got["n"][8:] == 0) and np.all(got["v_sum"][8:] == 0) and np.all(got["v2_sum"][8:] == 0)


def test_profile_errors():
    cfg = synth.base_config(L=(6, 6, 6), kT=1.0, seed=1)
    x, v, fl = synth.solvent(cfg, seed=1)
    s = api.System([dict(cfg=cfg, n=len(x))], "mixed", 64)
    s.set_state(0, x, v, fl)
    for bad in [dict(axis=3, n_bins=6), dict(axis=-1, n_bins=6), dict(axis=0, n_bins=0),
                dict(axis=0, n_bins=api.MAX_PROFILE_BINS + 1)]:
        with pytest.raises(api.RmpcdError):
            s.profile(0, **bad)
    with pytest.raises(api.RmpcdError):
        s.profile(1, 0, 6)
    _same(s.profile(0, 0, 6), _expect(s, 0, 0, 6))   # the system is still usable


def test_poiseuille_profile_from_the_kernel_matches_viscosity():
    """Mixed path, stick walls and body force g along x: the time-averaged
    v_x(z) from rmpcd_profile is the parabola g z (H - z) / (2 nu) with nu
    from the SRD closed form at the measured temperature (6 %), and the
    slab temperatures are flat."""
    H, g = 12, 0.005
    alpha = math.radians(130.0)
    cfg = synth.base_config(L=(24, 24, H), walls=1, rho_wall=10, g=(g, 0.0, 0.0), alpha=alpha, tau=1.0,
                            kT=1.0, seed=17, precision="mixed")
    x, v, fl = synth.solvent(cfg, seed=17)
    s = api.System([dict(cfg=cfg, n=len(x))], "mixed", 64)
    s.set_state(0, x, v, fl)
    s.step(150)
    acc = np.zeros((H, 3))
    cnt = np.zeros(H)
    T = np.zeros(H)
    temps = []
    for _ in range(250):
        s.step(1)
        p = s.profile(0, 2, H)
        acc += p["v_sum"]
        cnt += p["n"]
        T += orc.slab_fields(p)["T"]
        temps.append(s.observables(0)["temperature"])
    prof = acc[:, 0] / cnt
    z = np.arange(H) + 0.5
    shape = z * (H - z)
    a = (prof @ shape) / (shape @ shape)
    kTm = float(np.mean(temps))
    M = 10.0
    gm = M - 1.0 + math.exp(-M)
    nu = (kTm / 2.0 * (5.0 * M / (gm * (2.0 - math.cos(alpha) - math.cos(2 * alpha))) - 1.0)
          + (1.0 - math.cos(alpha)) / 18.0 * gm / M)
    assert abs(a - g / (2.0 * nu)) / (g / (2.0 * nu)) < 0.06, (a, g / (2 * nu))
    assert np.max(np.abs(prof - a * shape)) < 0.1 * a * shape.max()
    assert np.all(np.abs(acc[:, 1:] / cnt[:, None]) < 0.02)
    # slab temperatures (shear within a slab removed) agree with the cell estimator
    assert np.all(np.abs(T / 250 - kTm) < 0.03 * kTm)
