"""GPU parity of the rigid bead body (the Janus particle of §1.5): the CUDA
path through the C ABI against the FP64 oracle on the same seeded inputs.
FP64 path: solvent and body to the fp64 tolerance, species flags identical;
mixed path: within the mixed tolerance except for a few particles that
graze a cut-off.  Also batching, launch paths and the entry points' errors."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1608_04904_gb300 import api, build, synth
from parity_util import by_id, check_mixed_exceptions, near_boundary, pos_bad, pos_diff, vel_bad

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()


def _janus(precision, L=16, nb=120, seed=4, spin=40.0, frac_b=0.2, **kw):
    """A Janus particle slightly off the box centre, spun up so that it turns
    visibly within an interval; eps_B 1 on the catalytic hemisphere and 0.3
    on the other."""
    cfg = synth.base_config(L=(L, L, L), alpha=np.radians(130.0), tau=0.5, n_md=25, kT=1.0, seed=seed,
                            precision=precision, **kw)
    c = L / 2.0
    body = synth.janus_body(nb, (c + 0.3, c - 0.2, c + 0.1), seed=seed)
    body["eps_B"] = np.where(body["catalytic"] == 1, 1.0, 0.3)
    body["l"] = body["l"] * spin
    x, v, fl = synth.solvent(cfg, synth.body_exclusion(body), seed=seed + 1, frac_b=frac_b)
    return cfg, body, x, v, fl


def gpu(cfg, body, x, v, fl, precision, step=0, cap=64):
    s = api.System([dict(cfg=cfg, n=len(x), body=body)], precision, cap)
    s.set_state(0, x, v, fl)
    s.set_step(step)
    return s


def oracle(cfg, body, x, v, fl, step=0):
    return orc.OracleSystem(cfg, x, v, fl, body=body, step=step)


def _body_close(gb, ob, precision):
    if precision == "fp64":
        for k in ("x", "v", "q", "l"):
            ref = getattr(ob, k)
            assert np.allclose(gb[k], ref, rtol=1e-12, atol=1e-13 * max(1.0, np.abs(ref).max())), k
    else:
        assert np.allclose(gb["x"], ob.x, rtol=0, atol=1e-5)
        assert np.allclose(gb["v"], ob.v, rtol=0, atol=1e-5 * max(1.0, np.abs(ob.v).max()))
        assert np.allclose(gb["q"] * np.sign(gb["q"][0]), ob.q * np.sign(ob.q[0]), rtol=0, atol=1e-5)
        assert np.allclose(gb["l"], ob.l, rtol=0, atol=1e-4 * np.abs(ob.l).max())


@pytest.mark.parametrize("precision", PRECS)
def test_body_interval_parity(precision):
    cfg, body, x, v, fl = _janus(precision)
    g = gpu(cfg, body, x, v, fl, precision, step=3)
    g.stream_interval()
    st = g.get_state()
    o = oracle(cfg, body, x, v, fl, step=3)
    o.interval()
    assert o.near.sum() > 3000
    assert not np.allclose(o.body.q, body["q"], atol=1e-3)        # it turned
    assert (o.flags != fl).sum() > 0                              # catalysis happened
    pb = pos_bad(st["x"], o.x, cfg["L"], 0, precision)
    vb = vel_bad(st["v"], o.v, cfg["kT"], precision)
    if precision == "fp64":
        assert not pb.any() and not vb.any()
        assert np.array_equal(st["flags"], o.flags)
    else:
        fd = st["flags"] != o.flags
        near = o.near.astype(bool)
        check_mixed_exceptions(vb, near, fd, st["v"] - o.v, cfg["kT"], 2)
        check_mixed_exceptions(pb, near, fd, pos_diff(st["x"], o.x, cfg["L"], 0), cfg["kT"], 2, "position")
        assert fd.sum() <= 2
    _body_close(g.get_body(0), o.body, precision)


def _compare_step(cfg, st, o, precision):
    gid, gx, gv, gf, gc = by_id(st["id"], st["id"], st["x"], st["v"], st["flags"], st["cell"])
    oid, ox, ov, of, oc, onear = by_id(o.id, o.id, o.x, o.v, o.flags, o.key, o.near.astype(bool))
    assert np.array_equal(gid, oid)
    if precision == "fp64":
        assert np.array_equal(st["id"], o.id)
        assert np.array_equal(gc, oc)
        assert np.array_equal(gf, of)
        assert not pos_bad(gx, ox, cfg["L"], 0, "fp64").any()
        assert not vel_bad(gv, ov, cfg["kT"], "fp64").any()
        return
    mism = gc != oc
    border = near_boundary(ox, o.shift, 1e-4)
    assert np.all(border[mism]), "key mismatch away from a cell boundary"
    assert mism.sum() <= max(3, 1e-4 * len(gc))
    badcells = np.isin(oc, oc[mism]) | np.isin(oc, gc[mism])
    assert not pos_bad(gx, ox, cfg["L"], 0, "mixed").any()
    vb = vel_bad(gv, ov, cfg["kT"], "mixed") & ~badcells
    check_mixed_exceptions(vb, onear, gf != of, gv - ov, cfg["kT"], 2)
    assert (gf != of).sum() <= 2 + mism.sum()


@pytest.mark.parametrize("precision", PRECS)
def test_fused_step_parity_body(precision):
    cfg, body, x, v, fl = _janus(precision, seed=6, bulk_rate=0.05)
    g = gpu(cfg, body, x, v, fl, precision, step=7)
    g.step(1)
    o = oracle(cfg, body, x, v, fl, step=7)
    o.step(1)
    _compare_step(cfg, g.get_state(), o, precision)
    _body_close(g.get_body(0), o.body, precision)


def test_fused_three_steps_body_fp64():
    cfg, body, x, v, fl = _janus("fp64", L=20, nb=250, seed=8)
    g = gpu(cfg, body, x, v, fl, "fp64")
    g.step(3)
    o = oracle(cfg, body, x, v, fl)
    o.step(3)
    _compare_step(cfg, g.get_state(), o, "fp64")
    _body_close(g.get_body(0), o.body, "fp64")


@pytest.mark.parametrize("precision", PRECS)
def test_body_granular_equals_fused_and_graphs(precision):
    cfg, body, x, v, fl = _janus(precision, seed=9)
    a = gpu(cfg, body, x, v, fl, precision, step=2)
    a.step(2)
    b = gpu(cfg, body, x, v, fl, precision, step=2)
    for k in range(2):
        b.stream_interval()
        b.shift_and_sort()
        b.collide()
        b.react()
        b.set_step(3 + k)
    c = gpu(cfg, body, x, v, fl, precision, step=2)
    c.set_graphs(False)
    c.step(2)
    sa, sb, sc = a.get_state(), b.get_state(), c.get_state()
    for key in ("id", "x", "v", "flags", "cell"):
        assert np.array_equal(sa[key], sb[key]), key
        assert np.array_equal(sa[key], sc[key]), key
    for key in ("x", "v", "q", "l"):
        assert np.array_equal(a.get_body(0)[key], b.get_body(0)[key])
        assert np.array_equal(a.get_body(0)[key], c.get_body(0)[key])


@pytest.mark.parametrize("precision", PRECS)
def test_batch_of_bodies_equals_single_runs(precision):
    """Replicas of uneven sides and bead counts in one system (one launch per
    kernel) give bit-identical results to the same replicas run alone, and a
    replica without a body runs beside them unchanged."""
    reps = []
    for side, nb, seed in ((16, 100, 11), (20, 300, 12), (24, 173, 13)):
        cfg, body = synth.batch_janus(side, seed, precision=precision, nb=nb)
        x, v, fl = synth.solvent(cfg, synth.body_exclusion(body), seed=seed + 1)
        reps.append((cfg, body, x, v, fl))
    cfg0 = synth.base_config(L=(12, 12, 12), seed=14, precision=precision)
    x0, v0, f0 = synth.solvent(cfg0, seed=15)
    batch = api.System([dict(cfg=c, n=len(x), body=b) for c, b, x, v, f in reps] + [dict(cfg=cfg0, n=len(x0))],
                       precision, 0)
    for r, (c, b, x, v, f) in enumerate(reps):
        batch.set_state(r, x, v, f)
    batch.set_state(len(reps), x0, v0, f0)
    batch.step(3)
    for r, (c, b, x, v, f) in enumerate(reps):
        one = api.System([dict(cfg=c, n=len(x), body=b)], precision, batch.bucket_cap())
        one.set_state(0, x, v, f)
        one.step(3)
        s1, sb = one.get_state(0), batch.get_state(r)
        for key in ("id", "x", "v", "flags", "cell"):
            assert np.array_equal(s1[key], sb[key]), (r, key)
        for key in ("x", "v", "q", "l"):
            assert np.array_equal(one.get_body(0)[key], batch.get_body(r)[key]), (r, key)
    plain = api.System([dict(cfg=cfg0, n=len(x0))], precision, batch.bucket_cap())
    plain.set_state(0, x0, v0, f0)
    plain.step(3)
    for key in ("id", "x", "v", "flags"):
        assert np.array_equal(plain.get_state(0)[key], batch.get_state(len(reps))[key]), key


def test_batch_replica_at_full_size_matches_oracle():
    """The largest replica side of the batched ensemble (48, 1.1 M particles,
    300 beads) through the fused mixed path: one interval against the oracle
    on the body state and on a sample of particles near the body."""
    cfg, body = synth.batch_janus(48, 21, precision="mixed", nb=300)
    x, v, fl = synth.solvent(cfg, synth.body_exclusion(body), seed=22)
    g = gpu(cfg, body, x, v, fl, "mixed")
    g.step(1)
    o = oracle(cfg, body, x, v, fl)
    o.step(1)
    _body_close(g.get_body(0), o.body, "mixed")
    st = g.get_state()
    gid, gx, gv = by_id(st["id"], st["id"], st["x"], st["v"])
    oid, ox, ov = by_id(o.id, o.id, o.x, o.v)
    assert np.array_equal(gid, oid)
    assert pos_bad(gx, ox, cfg["L"], 0, "mixed").sum() <= 3


def test_body_entry_point_errors():
    cfg, body, x, v, fl = _janus("mixed")
    s = api.System([dict(cfg=cfg, n=len(x))], "mixed", 64)
    with pytest.raises(api.RmpcdError) as e:
        s.get_body(0)
    assert e.value.code == "EINVAL"
    bad = dict(body, b=body["b"] + 0.5)                      # not centred
    with pytest.raises(api.RmpcdError) as e:
        s.set_body(0, bad)
    assert e.value.code == "EINVAL"
    R = synth.fibonacci_sphere(40, 4.0)
    R[:, 0] *= 1.5                                           # ellipsoid ...
    th = 0.3
    rot = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    bad = dict(body, b=R @ rot.T - (R @ rot.T).mean(0), eps_A=1.0, eps_B=1.0, catalytic=0)   # ... turned off its axes
    with pytest.raises(api.RmpcdError) as e:
        s.set_body(0, bad)
    assert e.value.code == "EINVAL"
    with pytest.raises(api.RmpcdError):
        s.set_body(0, dict(body, q=np.array([1.0, 0.1, 0.0, 0.0])))     # not a unit quaternion
    with pytest.raises(api.RmpcdError):
        s.set_body(0, dict(body, b=np.zeros((0, 3)), eps_A=1.0, eps_B=1.0, catalytic=0))
    small = synth.base_config(L=(10, 10, 10), precision="mixed")
    t = api.System([dict(cfg=small, n=10)], "mixed", 64)
    with pytest.raises(api.RmpcdError):
        t.set_body(0, body)                                  # reach 5.1 does not fit a box of 10
    col = [dict(x=(8.0, 8.0, 8.0), v=(0.0, 0.0, 0.0), mass=100.0, sigma=2.0, eps_A=1.0, eps_B=1.0, catalytic=0)]
    u = api.System([dict(cfg=cfg, n=len(x), colloids=col)], "mixed", 64)
    with pytest.raises(api.RmpcdError):
        u.set_body(0, body)                                  # a replica has colloids or a body
    s.set_body(0, body)                                      # the valid body is accepted
    gb = s.get_body(0)
    assert np.array_equal(gb["x"], body["x"]) and np.array_equal(gb["q"], body["q"])


def test_body_skin_violation_is_reported():
    cfg, body, x, v, fl = _janus("fp64", skin=0.05)
    body["v"] = np.array([0.5, 0.0, 0.0])                    # 0.25 per interval > skin
    g = gpu(cfg, body, x, v, fl, "fp64")
    with pytest.raises(api.RmpcdError) as e:
        g.step(1)
        g.sync()
    assert e.value.code == "ESKIN"
