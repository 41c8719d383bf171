"""GPU parity in compact Hilbert cell order (rmpcd_set_cell_order): fused
steps against the oracle run in the same order on the FP64 path (storage
order by (Hilbert rank, id), keys and flags identical; positions and
velocities within the FP64 tolerance); the mixed path in Hilbert order
equal by id, bit for bit, to the mixed path in linear order; and a switch
of order in the middle of a run."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1608_04904_gb300 import api, build, synth
from parity_util import by_id, compare_step, pos_bad, vel_bad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()


def _setup(name, precision):
    """(cfg, replica kwargs, oracle kwargs, x, v, flags)."""
    if name == "dimer_slabs_bulk":
        cfg, col, bonds = synth.dimer32(precision=precision, seed=31, L=16)
        cfg = dict(cfg, slabs=[(0.0, 3.0, 0.45), (8.0, 11.0, 0.25)], bulk_rate=0.05)
        x, v, f = synth.solvent(cfg, col, seed=32, frac_b=0.3)
        return cfg, dict(colloids=col, bonds=bonds), dict(colloids=synth.colloid_arrays(col), bonds=bonds), x, v, f
    if name == "channel":
        cfg = synth.base_config(L=(20, 12, 10), walls=1, rho_wall=10, g=(0.002, 0.0, 0.0), tau=1.0, seed=33,
                                precision=precision, bulk_rate=0.02)
        x, v, f = synth.solvent(cfg, seed=34, frac_b=0.4)
        return cfg, {}, {}, x, v, f
    if name == "janus":
        cfg, body = synth.batch_janus(16, 35, precision=precision, nb=120)
        x, v, f = synth.solvent(cfg, synth.body_exclusion(body), seed=36, frac_b=0.2)
        return cfg, dict(body=body), dict(body=body), x, v, f
    raise ValueError(name)


@pytest.mark.parametrize("name", ["dimer_slabs_bulk", "channel", "janus"])
def test_fp64_fused_steps_in_hilbert_order_equal_the_oracle(name):
    cfg, rk, ok, x, v, f = _setup(name, "fp64")
    s = api.System([dict(cfg=cfg, n=len(x), **rk)], "fp64", 0)
    s.set_cell_order("hilbert")
    assert s.get_cell_order() == "hilbert"
    s.set_state(0, x, v, f)
    s.set_step(5)
    o = orc.OracleSystem(cfg, x, v, f, step=5, cell_order="hilbert", **ok)
    for _ in range(3):
        s.step(1)
        o.step(1)
        st = s.get_state(0)
        compare_step(cfg, st, o, "fp64")
        # storage runs by Hilbert rank of the cell key, then id
        r = o.rank[st["cell"]]
        assert np.all(np.diff(r) >= 0)
    s.close()


@pytest.mark.parametrize("name", ["dimer_slabs_bulk", "channel", "janus"])
def test_mixed_hilbert_order_equals_linear_order_by_id(name):
    cfg, rk, ok, x, v, f = _setup(name, "mixed")
    runs = []
    for order in ("linear", "hilbert"):
        s = api.System([dict(cfg=cfg, n=len(x), **rk)], "mixed", 0)
        s.set_cell_order(order)
        s.set_state(0, x, v, f)
        s.step(4)
        st = s.get_state(0)
        runs.append(by_id(st["id"], st["x"], st["v"], st["flags"], st["cell"]))
        s.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_switching_order_in_a_run():
    cfg, rk, ok, x, v, f = _setup("dimer_slabs_bulk", "fp64")
    s = api.System([dict(cfg=cfg, n=len(x), **rk)], "fp64", 0)
    s.set_state(0, x, v, f)
    o = orc.OracleSystem(cfg, x, v, f, **ok)
    s.step(2)
    o.step(2)
    s.set_cell_order("hilbert")
    s.step(2)
    o.step(2)
    st = s.get_state(0)
    gid, gx, gv, gf = by_id(st["id"], st["id"], st["x"], st["v"], st["flags"])
    oid, ox, ov, of = by_id(o.id, o.id, o.x, o.v, o.flags)
    assert np.array_equal(gid, oid) and np.array_equal(gf, of)
    assert not pos_bad(gx, ox, cfg["L"], cfg.get("walls", 0), "fp64").any()
    assert not vel_bad(gv, ov, cfg["kT"], "fp64").any()
    s.set_cell_order("linear")
    s.step(1)
    o.step(1)
    compare_step(cfg, s.get_state(0), o, "fp64")
    with pytest.raises(KeyError):
        s.set_cell_order("morton")
    s.close()
