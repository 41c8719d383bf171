"""The oracle's OpenMP loops (per particle and per cell; colloid and body
force totals in exact 64-bit fixed point) give bit-identical results for any
thread count."""
import math

import numpy as np
import pytest

from paper_1608_04904_gb300 import synth


def _run(orc, threads, make, steps):
    orc.set_threads(threads)
    try:
        s = make()
        s.step(steps)
        return s
    finally:
        orc.set_threads(1)


def _same(a, b):
    assert np.array_equal(a.id, b.id)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and np.array_equal(a.flags, b.flags)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.V, b.V)


def test_threads_all_cores_available(orc):
    n = orc.set_threads(0)
    orc.set_threads(1)
    assert n >= 1 and orc.get_threads() == 1


def test_dimer_with_reactions_is_thread_count_independent(orc):
    cfg, col, bonds = synth.dimer32(precision="fp64", L=12)
    cfg["bulk_rate"] = 0.05
    x, v, fl = synth.solvent(cfg, col, seed=8)
    make = lambda: orc.OracleSystem(cfg, x, v, fl, colloids=synth.colloid_arrays(col), bonds=bonds)
    _same(_run(orc, 1, make, 3), _run(orc, 4, make, 3))


def test_walls_slabs_and_lj_colloids_are_thread_count_independent(orc):
    cfg = synth.base_config(L=(16, 8, 8), walls=1, rho_wall=10, g=(0.002, 0.0, 0.0), bulk_rate=0.1,
                            slabs=[(0.0, 3.0, 1.3)], cc_lj=(1.0, 3.0, 7.5), seed=4)
    col = [dict(x=(4.0, 4.0, 4.0), v=(0.1, 0.0, 0.0), mass=80.0, sigma=1.5, eps_A=1.0, eps_B=1.0, catalytic=1),
           dict(x=(10.0, 4.0, 4.0), v=(-0.1, 0.0, 0.0), mass=80.0, sigma=1.5, eps_A=1.0, eps_B=0.5, catalytic=0)]
    x, v, fl = synth.solvent(cfg, col, seed=9, frac_b=0.3)
    make = lambda: orc.OracleSystem(cfg, x, v, fl, colloids=synth.colloid_arrays(col))
    _same(_run(orc, 1, make, 3), _run(orc, 3, make, 3))


def test_rigid_body_is_thread_count_independent(orc):
    cfg, body = synth.batch_janus(14, 3, precision="fp64", nb=100)
    x, v, fl = synth.solvent(cfg, synth.body_exclusion(body), seed=6)
    make = lambda: orc.OracleSystem(cfg, x, v, fl, body=body)
    a, b = _run(orc, 1, make, 2), _run(orc, 4, make, 2)
    _same(a, b)
    assert np.array_equal(a.body.q, b.body.q) and np.array_equal(a.body.x, b.body.x)
