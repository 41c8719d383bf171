"""Pins of the oracle's species reservoirs (the chemotactic set-up of §1.5:
a Poiseuille flow with a two-species gradient across it): after a step the
reservoir cells are pure and nothing else changed species; in steady state
the B fraction between the reservoirs is the linear profile of 1-D diffusion
with fixed end concentrations, while the channel flow runs across it."""
import numpy as np

from paper_1608_04904_gb300 import synth


def _cfg(**kw):
    return synth.base_config(L=(8, 16, 6), walls=1, rho_wall=10, g=(0.005, 0.0, 0.0),
                             alpha=np.radians(130.0), tau=0.5, kT=1.0, seed=21,
                             reservoirs=((0, 2), (14, 16)), **kw)


def test_reservoir_cells_are_pure_after_a_step(orc):
    cfg = _cfg()
    x, v, fl = synth.solvent(cfg, seed=22, frac_b=0.5)
    o = orc.OracleSystem(cfg, x, v, fl)
    o.interval()
    o.shift_and_sort()
    before = o.flags.copy()
    o.collide()
    o.react()
    o.reservoirs()
    cy = (o.key // cfg["L"][0]) % cfg["L"][1]
    a = (cy >= 0) & (cy < 2)
    b = (cy >= 14) & (cy < 16)
    assert a.sum() > 100 and b.sum() > 100
    assert np.all(o.flags[a] == 0) and np.all(o.flags[b] == 1)
    assert np.array_equal(o.flags[~a & ~b], before[~a & ~b])


def test_steady_gradient_is_linear_between_the_reservoirs(orc):
    """After relaxation the time-averaged B fraction in the y slabs between
    the layers rises linearly from about 0 to about 1; the fitted slope in the
    interior is 1 / 12 per cell within 15 %, and the flow along x is there."""
    cfg = _cfg()
    x, v, fl = synth.solvent(cfg, seed=23)
    o = orc.OracleSystem(cfg, x, v, fl)
    o.step(300)
    nb = np.zeros(16)
    n = np.zeros(16)
    vx = 0.0
    for _ in range(300):
        o.step(1)
        p = orc.slab_profile(16, o.x[:, 1], o.v, o.flags, 16)
        nb += p["n_B"]
        n += p["n"]
        vx += o.v[:, 0].mean()
    c = nb / n
    y = np.arange(16) + 0.5
    inner = (y > 3) & (y < 13)
    slope, icpt = np.polyfit(y[inner], c[inner], 1)
    assert abs(slope - 1.0 / 12.0) < 0.15 / 12.0, slope
    assert np.all(np.diff(c[2:14]) > -0.02)           # monotone up to noise
    # y in [1, 2) always lies in the A layer and [15, 16) in the B layer of
    # the shifted grid; [0, 1) falls in column 15 (B) whenever y < the shift
    assert c[1] < 0.05 and c[15] > 0.95 and 0.3 < c[0] < 0.7
    assert vx / 300 > 0.005                           # the channel flows
