"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Integer results (cell keys, sort permutation, species
flags) must be bit-identical; velocities and positions within the
tolerances of parity_util (fp64 1e-12, mixed 1e-5)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1608_04904_gb300 import api, build, synth
from parity_util import (by_id, check_mixed_exceptions, compare_step as _compare_step, near_boundary, pos_bad,
                         pos_diff, vel_bad)

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()


def gpu(cfg, x, v, fl, col=(), bonds=(), precision="fp64", cap=64, step=0):
    s = api.System.single(cfg, len(x), col, bonds, precision=precision, bucket_cap=cap)
    s.set_state(0, x, v, fl)
    s.set_step(step)
    return s


def oracle(cfg, x, v, fl, col=(), bonds=(), step=0):
    return orc.OracleSystem(cfg, x, v, fl, colloids=synth.colloid_arrays(col) if col else None,
                            bonds=list(bonds), step=step)


SORT_CASES = {
    "ragged": dict(L=(5, 7, 6), n=2113),
    "rho10": dict(L=(16, 16, 16), n=40960),
    "walls": dict(L=(8, 8, 6), n=3000, walls=1, rho_wall=10),
    "long": dict(L=(40, 8, 9), n=29000),
}


def _case(name, precision, seed=3, **extra):
    c = dict(SORT_CASES[name])
    n = c.pop("n")
    cfg = synth.base_config(precision=precision, seed=seed, **c, **extra)
    x, v, fl = synth.solvent(cfg, n=n, seed=seed + 100, frac_b=0.3)
    return cfg, x, v, fl


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name", list(SORT_CASES))
def test_shift_and_sort_bit_exact(precision, name):
    cfg, x, v, fl = _case(name, precision)
    g = gpu(cfg, x, v, fl, precision=precision, step=7)
    g.shift_and_sort()
    st = g.get_state()
    o = oracle(cfg, x, v, fl, step=7)
    o.shift_and_sort()
    assert np.array_equal(st["id"], o.id)
    assert np.array_equal(st["cell"], o.key)
    assert np.array_equal(st["flags"], o.flags)
    assert np.array_equal(st["x"], o.x)
    assert np.array_equal(st["v"], o.v)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name,extra", [
    ("ragged", {}), ("rho10", {}), ("long", {"alpha": math.radians(90.0)}),
    ("walls", {}), ("rho10", {"slabs": [(0.0, 4.0, 1.5), (8.0, 10.0, 0.5)]}),
])
def test_collide_parity(precision, name, extra):
    cfg, x, v, fl = _case(name, precision, **extra)
    g = gpu(cfg, x, v, fl, precision=precision, step=11)
    g.shift_and_sort()
    g.collide()
    st = g.get_state()
    o = oracle(cfg, x, v, fl, step=11)
    o.shift_and_sort()
    o.collide()
    assert np.array_equal(st["id"], o.id)
    bad = vel_bad(st["v"], o.v, cfg["kT"], precision)
    assert not bad.any(), (int(bad.sum()), np.abs(st["v"] - o.v).max())


def test_fp64_srd_is_bit_exact():
    cfg, x, v, fl = _case("rho10", "fp64")
    g = gpu(cfg, x, v, fl, precision="fp64", step=2)
    g.shift_and_sort()
    g.collide()
    o = oracle(cfg, x, v, fl, step=2)
    o.shift_and_sort()
    o.collide()
    assert np.array_equal(g.get_state()["v"], o.v)


@pytest.mark.parametrize("precision", PRECS)
def test_single_particle_wall_cells_collide(precision):
    """A dilute channel (about two particles per cell) puts many wall cells at
    one real particle; each collides with rho_wall - 1 virtual partners (§1.4),
    on the GPU as in the oracle (the virtual momentum's Gaussian goes through
    log, sqrt and sincos, so fp64 agrees to their last bits, not bit for bit)."""
    cfg = synth.base_config(L=(8, 8, 6), walls=1, rho_wall=10, precision=precision, seed=21)
    x, v, fl = synth.solvent(cfg, n=800, seed=121)
    g = gpu(cfg, x, v, fl, precision=precision, step=5)
    g.shift_and_sort()
    g.collide()
    st = g.get_state()
    o = oracle(cfg, x, v, fl, step=5)
    o.shift_and_sort()
    v_sorted = o.v.copy()
    o.collide()
    # the case exercises the rule: lone particles in wall layers that moved
    nz = cfg["L"][2] + 1
    layer = o.key // (cfg["L"][0] * cfg["L"][1])
    lone = (o.count[o.key] == 1) & ((layer == 0) | (layer == nz - 1))
    assert lone.sum() >= 10 and np.all(np.any(o.v[lone] != v_sorted[lone], axis=1))
    assert np.array_equal(st["id"], o.id)
    bad = vel_bad(st["v"], o.v, cfg["kT"], precision)
    assert not bad.any(), (int(bad.sum()), np.abs(st["v"] - o.v).max())


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("rate", [0.05, 1e6])
def test_bulk_reaction_flags_bit_exact(precision, rate):
    cfg, x, v, fl = _case("rho10", precision, bulk_rate=rate)
    x, v, fl = synth.solvent(cfg, n=len(x), seed=5, frac_b=0.5, tag_frac=0.2)
    g = gpu(cfg, x, v, fl, precision=precision, step=4)
    g.shift_and_sort()
    g.react()
    st = g.get_state()
    o = oracle(cfg, x, v, fl, step=4)
    o.shift_and_sort()
    o.react()
    assert np.array_equal(st["id"], o.id)
    assert np.array_equal(st["flags"], o.flags)
    assert (st["flags"] & 1).sum() < (fl & 1).sum()


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("kind", ["periodic_g", "walls_g"])
def test_free_flight_parity(precision, kind):
    if kind == "periodic_g":
        cfg = synth.base_config(L=(9, 10, 11), g=(0.01, -0.003, 0.002), tau=0.7, precision=precision)
    else:
        cfg = synth.base_config(L=(8, 8, 10), walls=1, rho_wall=10, g=(0.02, 0.0, 0.0), tau=1.0,
                                precision=precision)
    x, v, fl = synth.solvent(cfg, n=9000, seed=8)
    g = gpu(cfg, x, v, fl, precision=precision)
    g.stream_interval()
    st = g.get_state()
    o = oracle(cfg, x, v, fl)
    o.interval()
    assert np.array_equal(st["id"], np.arange(len(x)))
    assert not pos_bad(st["x"], o.x, cfg["L"], cfg["walls"], precision).any()
    assert not vel_bad(st["v"], o.v, cfg["kT"], precision).any()
    if kind == "walls_g":
        assert st["x"][:, 2].min() >= 0.0 and st["x"][:, 2].max() <= cfg["L"][2]
        assert (np.sign(st["v"][:, 2]) != np.sign(v[:, 2])).sum() > 100


def _dimer(precision, L=12, seed=2, **kw):
    cfg, col, bonds = synth.dimer32(precision=precision, L=L)
    cfg.update(kw)
    x, v, fl = synth.solvent(cfg, col, seed=seed, frac_b=0.2, tag_frac=0.0)
    return cfg, col, bonds, x, v, fl


@pytest.mark.parametrize("precision", PRECS)
def test_md_interval_parity(precision):
    cfg, col, bonds, x, v, fl = _dimer(precision)
    col[0]["v"] = (0.02, -0.01, 0.0)
    col[1]["v"] = (0.02, -0.01, 0.0)
    g = gpu(cfg, x, v, fl, col, bonds, precision=precision, step=3)
    g.stream_interval()
    st = g.get_state()
    o = oracle(cfg, x, v, fl, col, bonds, step=3)
    o.interval()
    near = o.near.astype(bool)
    assert near.sum() > 500
    pb = pos_bad(st["x"], o.x, cfg["L"], 0, precision)
    vb = vel_bad(st["v"], o.v, cfg["kT"], precision)
    if precision == "fp64":
        assert not pb.any() and not vb.any()
        assert np.array_equal(st["flags"], o.flags)
    else:
        # FP32 forces: a particle that grazes a cut-off may take the other branch
        fd = st["flags"] != o.flags
        check_mixed_exceptions(vb, near, fd, st["v"] - o.v, cfg["kT"], 2)
        check_mixed_exceptions(pb, near, fd, pos_diff(st["x"], o.x, cfg["L"], 0), cfg["kT"], 2, "position")
        assert fd.sum() <= 2
    gc = g.get_colloids(0)
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.allclose(gc["x"], o.X, rtol=0, atol=tol * cfg["L"][0])
    assert np.allclose(gc["v"], o.V, rtol=0, atol=max(tol, 1e-9) * 10)
    r = gc["x"][0] - gc["x"][1]
    # exact RATTLE: to rounding of the path's precision
    assert abs(np.linalg.norm(r) - 4.5) < (1e-11 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", PRECS)
def test_fused_step_parity_dimer(precision):
    cfg, col, bonds, x, v, fl = _dimer(precision, bulk_rate=0.05)
    g = gpu(cfg, x, v, fl, col, bonds, precision=precision, step=5)
    g.step(1)
    o = oracle(cfg, x, v, fl, col, bonds, step=5)
    o.step(1)
    _compare_step(cfg, g.get_state(), o, precision)
    assert g.get_step() == 6


def test_fused_three_steps_fp64():
    cfg, col, bonds, x, v, fl = _dimer("fp64", L=14, bulk_rate=0.05)
    g = gpu(cfg, x, v, fl, col, bonds, precision="fp64")
    g.step(3)
    o = oracle(cfg, x, v, fl, col, bonds)
    o.step(3)
    _compare_step(cfg, g.get_state(), o, "fp64")
    gc = g.get_colloids(0)
    assert np.allclose(gc["x"], o.X, rtol=0, atol=1e-10)


@pytest.mark.parametrize("precision", PRECS)
def test_fused_equals_granular(precision):
    cfg, col, bonds, x, v, fl = _dimer(precision, bulk_rate=0.05)
    a = gpu(cfg, x, v, fl, col, bonds, precision=precision, step=9)
    a.step(2)
    sa = a.get_state()
    b = gpu(cfg, x, v, fl, col, bonds, precision=precision, step=9)
    for k in range(2):
        b.stream_interval()
        b.shift_and_sort()
        b.collide()
        b.react()
        b.set_step(10 + k)
    sb = b.get_state()
    for key in ("id", "x", "v", "flags", "cell"):
        assert np.array_equal(sa[key], sb[key]), key
    assert np.array_equal(a.get_colloids(0)["x"], b.get_colloids(0)["x"])


@pytest.mark.parametrize("precision", PRECS)
def test_runs_are_deterministic(precision):
    cfg, col, bonds, x, v, fl = _dimer(precision, bulk_rate=0.05)
    outs = []
    for _ in range(2):
        g = gpu(cfg, x, v, fl, col, bonds, precision=precision)
        g.step(3)
        outs.append(g.get_state())
    for key in outs[0]:
        assert np.array_equal(outs[0][key], outs[1][key]), key


@pytest.mark.parametrize("precision", PRECS)
def test_observables_match_oracle(precision):
    cfg, col, bonds, x, v, fl = _dimer(precision, bulk_rate=0.05)
    g = gpu(cfg, x, v, fl, col, bonds, precision=precision)
    g.step(2)
    ob = g.observables(0)
    o = oracle(cfg, x, v, fl, col, bonds)
    o.step(2)
    tol = 1e-10 if precision == "fp64" else 2e-5
    assert abs(ob["temperature"] - o.temperature()) < tol * o.temperature()
    assert ob["n_B"] == int((o.flags & 1).sum()) or precision == "mixed"
    assert ob["n_solvent"] == len(x)
    assert np.allclose(ob["momentum"], o.v.sum(0), rtol=0, atol=1e-6 if precision == "fp64" else 1e-2)
    # granular path computes the same numbers on the same grid
    st = g.get_state()
    h = gpu(cfg, st["x"], st["v"], st["flags"], col, bonds, precision=precision, step=1)
    h.shift_and_sort()
    assert abs(h.observables(0)["temperature"] - ob["temperature"]) < 1e-6 * ob["temperature"]


def test_empty_and_single_particle_systems():
    for n in (0, 1):
        cfg = synth.base_config(L=(4, 5, 6), precision="mixed")
        x, v, fl = synth.solvent(cfg, n=n, seed=1)
        g = gpu(cfg, x, v, fl, precision="mixed")
        g.step(3)
        st = g.get_state()
        assert len(st["id"]) == n
        o = oracle(cfg, x, v, fl)
        o.step(3)
        if n:
            assert not pos_bad(st["x"], o.x, cfg["L"], 0, "mixed").any()
            assert np.array_equal(st["v"], o.v.astype(np.float32).astype(np.float64)) or \
                not vel_bad(st["v"], o.v, 1.0, "mixed").any()


@pytest.mark.parametrize("precision", PRECS)
def test_one_crowded_cell(precision):
    cfg = synth.base_config(L=(4, 4, 4), precision=precision, bulk_rate=0.3)
    rng = np.random.Generator(np.random.PCG64(4))
    n = 700
    x = 1.25 + np.floor(rng.uniform(0, 0.5, (n, 3)) * 2**24) * 2.0**-24
    v = rng.standard_normal((n, 3)).astype(np.float32).astype(np.float64)
    fl = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    g = gpu(cfg, x, v, fl, precision=precision, cap=768)
    g.shift_and_sort()
    g.collide()
    g.react()
    st = g.get_state()
    o = oracle(cfg, x, v, fl)
    o.shift_and_sort()
    o.collide()
    o.react()
    assert o.count.max() > 300
    assert np.array_equal(st["id"], o.id)
    assert np.array_equal(st["flags"], o.flags)
    assert not vel_bad(st["v"], o.v, 1.0, precision).any()


@pytest.mark.parametrize("precision", PRECS)
def test_overflow_list_keeps_fused_steps_exact(precision):
    """A cell row of 16 at density 10: a few per cent of the cells spill into
    the overflow list every collision, and a crowd of 300 particles puts a few
    cells far past the row.  The cell pass reads the spilled records back in
    canonical order: fused steps equal the oracle (fp64 bit for bit) and no
    EOVERFLOW is raised."""
    if precision == "fp64":
        # the sphere dimer: the MD kernel bins its near particles too
        cfg, col, bonds, x, v, fl = _dimer(precision, bulk_rate=0.05)
    else:
        # no colloids: the FP32 MD's few exceptions of the tolerance, which
        # the crowd would multiply, stay out of this test of the binning
        cfg = synth.base_config(L=(12, 12, 12), precision=precision, bulk_rate=0.05, seed=6)
        col, bonds = [], []
        x, v, fl = synth.solvent(cfg, seed=7, frac_b=0.2)
    x = x.copy()
    rng = np.random.Generator(np.random.PCG64(12))
    x[:300] = 1.25 + np.floor(rng.uniform(0.0, 0.5, (300, 3)) * 2**24) * 2.0**-24
    g = gpu(cfg, x, v, fl, col, bonds, precision=precision, cap=16, step=5)
    o = oracle(cfg, x, v, fl, col, bonds, step=5)
    for k in range(3):
        g.step(1)
        o.step(1)
        if k == 0:
            assert o.count.max() > 32 and (o.count > 16).sum() > 10
        _compare_step(cfg, g.get_state(), o, precision)
    assert g.bucket_cap() == 16


def test_bucket_overflow_is_reported():
    """EOVERFLOW remains for a cell beyond what the cell pass stages (1536
    particles) and for a full overflow list."""
    cfg = synth.base_config(L=(4, 4, 4), precision="mixed")
    n = 1600
    x = np.full((n, 3), 1.5) + np.linspace(0, 0.01, n)[:, None]
    v = np.zeros((n, 3))
    g = gpu(cfg, x, v, None, precision="mixed", cap=64)
    g.shift_and_sort()
    with pytest.raises(api.RmpcdError) as e:
        g.get_state()
    assert e.value.code == "EOVERFLOW"
    o = oracle(cfg, x, v, None)
    o.shift_and_sort()
    assert o.count.max() > 1536
    # a one-entry row: nearly every particle spills, past the list's 1024 + n/16 entries
    cfg = synth.base_config(L=(8, 8, 8), precision="mixed", seed=2)
    x, v, fl = synth.solvent(cfg, seed=3)
    g = gpu(cfg, x, v, fl, precision="mixed", cap=1)
    g.shift_and_sort()
    with pytest.raises(api.RmpcdError) as e:
        g.get_state()
    assert e.value.code == "EOVERFLOW"


def test_skin_violation_is_reported():
    cfg, col, bonds, x, v, fl = _dimer("fp64")
    col[0]["v"] = (3.0, 0.0, 0.0)
    col[1]["v"] = (3.0, 0.0, 0.0)
    g = gpu(cfg, x, v, fl, col, bonds, precision="fp64")
    g.stream_interval()
    with pytest.raises(api.RmpcdError) as e:
        g.sync()
    assert e.value.code == "ESKIN"


@pytest.mark.parametrize("precision", PRECS)
def test_replicas_in_one_batch_match_single_runs(precision):
    reps = []
    for k, L in enumerate((6, 9, 12)):
        cfg, col, bonds = synth.dimer32(precision=precision, L=L, seed=20 + k) if L == 12 else \
            (synth.base_config(L=(L, L + 1, L), precision=precision, seed=20 + k, bulk_rate=0.1), [], [])
        x, v, fl = synth.solvent(cfg, col, seed=30 + k, frac_b=0.3)
        reps.append((cfg, col, bonds, x, v, fl))
    b = api.System([dict(cfg=c, n=len(x), colloids=col, bonds=bd) for c, col, bd, x, v, fl in reps],
                   precision=precision)
    for r, (c, col, bd, x, v, fl) in enumerate(reps):
        b.set_state(r, x, v, fl)
    b.step(2)
    for r, (c, col, bd, x, v, fl) in enumerate(reps):
        s = gpu(c, x, v, fl, col, bd, precision=precision)
        s.step(2)
        sa, sb = b.get_state(r), s.get_state(0)
        for key in sa:
            assert np.array_equal(sa[key], sb[key]), (r, key)
        o = oracle(c, x, v, fl, col, bd)
        o.step(2)
        if precision == "fp64":
            _compare_step(c, sa, o, "fp64")


def test_device_pointer_state_roundtrip():
    import torch
    cfg, x, v, fl = _case("ragged", "fp64")
    g = api.System.single(cfg, len(x), precision="fp64")
    g.set_state(0, torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), torch.from_numpy(fl).cuda())
    out = {"x": torch.empty((len(x), 3), dtype=torch.float64, device="cuda"),
           "v": torch.empty((len(x), 3), dtype=torch.float64, device="cuda"),
           "flags": torch.empty(len(x), dtype=torch.uint8, device="cuda")}
    g.get_state(0, out=out)
    assert np.array_equal(out["x"].cpu().numpy(), x)
    assert np.array_equal(out["v"].cpu().numpy(), v)
    assert np.array_equal(out["flags"].cpu().numpy(), fl)


@pytest.mark.parametrize("precision", PRECS)
def test_md_launch_choices_do_not_change_results(precision):
    """The colloid forces are exact fixed-point sums, so every MD kernel and
    cluster size (and the autotuned choice) gives bit-identical states."""
    cfg, col, bonds, x, v, fl = _dimer(precision, bulk_rate=0.05)
    ref = None
    for kern in (1, 2, 3):
        for cs in (1, 2, 4, 8, 16, 0):
            if kern == 3 and cs > 1:
                continue   # the wide kernel takes no cluster size
            g = gpu(cfg, x, v, fl, col, bonds, precision=precision)
            try:
                g.set_tuning(cs, kern)
            except api.RmpcdError:
                # 16-CTA clusters: few-colloid kernel on capable devices only;
                # the wide kernel: mixed path only
                assert cs == 16 or (kern == 3 and precision == "fp64")
                continue
            g.step(14 if cs == 0 else 3)
            if cs == 0:
                assert g.get_tuning()[0] in (1, 2, 4, 8, 16) and g.get_tuning()[1] == kern
                continue
            st = g.get_state()
            cx = g.get_colloids(0)["x"]
            if ref is None:
                ref = (st, cx)
            else:
                for key in st:
                    assert np.array_equal(st[key], ref[0][key]), (kern, cs, key)
                assert np.array_equal(cx, ref[1])


def test_wide_md_kernel_matches_general_many_colloids():
    """Six spheres with colloid-colloid LJ (mixed path): the wide cooperative
    MD kernel gives the general kernel's states bit for bit."""
    cfg = synth.base_config(L=(48, 32, 32), alpha=np.radians(130.0), tau=0.5, n_md=20, kT=1.0,
                            cc_lj=(1.0, 3.0, 7.5), seed=7, precision="mixed")
    rng = np.random.Generator(np.random.PCG64(8))
    pos = [(8.0, 8.0, 8.0), (16.0, 9.0, 9.0), (30.0, 20.0, 12.0), (38.0, 24.0, 20.0), (10.0, 24.0, 24.0),
           (24.0, 16.0, 26.0)]
    col = [dict(x=p, v=tuple(rng.normal(0.0, 0.05, 3)), mass=120.0, sigma=2.0, eps_A=1.0, eps_B=0.5,
                catalytic=int(k % 2)) for k, p in enumerate(pos)]
    x, v, fl = synth.solvent(cfg, col, seed=9, frac_b=0.2)
    out = []
    for kern in (1, 3):
        g = gpu(cfg, x, v, fl, col, [], precision="mixed")
        g.set_tuning(1 if kern == 1 else 0, kern)
        g.step(3)
        out.append((g.get_state(), g.get_colloids(0)))
    for key in out[0][0]:
        assert np.array_equal(out[0][0][key], out[1][0][key]), key
    assert np.array_equal(out[0][1]["x"], out[1][1]["x"])
    assert np.array_equal(out[0][1]["v"], out[1][1]["v"])


@pytest.mark.parametrize("precision", PRECS)
def test_graph_replay_equals_direct_launches(precision):
    """Intervals replayed from captured CUDA graphs (device-resident step)
    give the same states as direct launches, also across rmpcd_set_step."""
    import torch
    cfg, col, bonds, x, v, fl = _dimer(precision, bulk_rate=0.05)
    outs = []
    for graphs in (True, False):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            g = api.System.single(cfg, len(x), col, bonds, precision=precision, stream=stream)
            g.set_graphs(graphs)
            g.set_tuning(2, 0)
            g.set_state(0, x, v, fl)
            g.step(3)
            g.set_step(40)
            g.step(2)
            assert g.get_step() == 42
            outs.append((g.get_state(), g.get_colloids(0)["x"], g.observables(0)["temperature"]))
            g.close()
    for key in outs[0][0]:
        assert np.array_equal(outs[0][0][key], outs[1][0][key]), key
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_automatic_bucket_width():
    """bucket_cap = 0: the width follows the density, grows on a crowded
    start, and the run equals one with a fixed wide bucket."""
    cfg = synth.base_config(L=(16, 16, 16), precision="mixed", seed=3)
    x, v, fl = synth.solvent(cfg, seed=4)
    g = api.System.single(cfg, len(x), precision="mixed", bucket_cap=0)
    cap0 = g.bucket_cap()
    assert 16 <= cap0 <= 64 and cap0 % 8 == 0
    g.close()
    # 300 of the particles start in one cell
    x = x.copy()
    x[:300] = 5.0 + np.floor(np.random.default_rng(5).uniform(0.0, 1.0, (300, 3)) * 2**24) * 2.0**-24
    runs = []
    for cap in (0, 768):
        g = api.System.single(cfg, len(x), precision="mixed", bucket_cap=cap)
        g.set_state(0, x, v, fl)
        g.step(2)
        runs.append((g.get_state(), g.bucket_cap()))
        g.close()
    assert runs[0][1] > cap0   # the shifted grid splits the crowd over up to 8 cells
    for key in runs[0][0]:
        assert np.array_equal(runs[0][0][key], runs[1][0][key]), key


@pytest.mark.parametrize("precision", PRECS)
def test_chemotactic_reservoirs_in_the_cell_pass(precision):
    """The chemotactic set-up (§1.5 chemotactic_cell): a Poiseuille channel
    whose y columns [0, 2) and [14, 16) of the collision grid are species
    reservoirs (A and B).  Fused steps equal the oracle's (fp64 bit for bit,
    species flags bit-exact on both paths), and after each step the
    reservoir cells are pure."""
    cfg = synth.base_config(L=(8, 16, 6), walls=1, rho_wall=10, g=(0.005, 0.0, 0.0), alpha=math.radians(130.0),
                            tau=0.5, kT=1.0, seed=21, bulk_rate=0.02, reservoirs=((0, 2), (14, 16)),
                            precision=precision)
    x, v, fl = synth.solvent(cfg, seed=22, frac_b=0.5)
    g = gpu(cfg, x, v, fl, precision=precision, step=3)
    o = oracle(cfg, x, v, fl, step=3)
    for _ in range(3):
        g.step(1)
        o.step(1)
        st = g.get_state()
        _compare_step(cfg, st, o, precision)
        gid, gf = by_id(st["id"], st["id"], st["flags"])
        oid, of = by_id(o.id, o.id, o.flags)
        assert np.array_equal(gf, of)
        cy = (st["cell"] // cfg["L"][0]) % cfg["L"][1]
        assert np.all(st["flags"][(cy >= 0) & (cy < 2)] == 0)
        assert np.all(st["flags"][(cy >= 14) & (cy < 16)] == 1)
    assert ((st["flags"] & 1) == 1).sum() > 0.2 * len(x)



@pytest.mark.parametrize("precision", PRECS)
def test_md_substeps_equal_the_interval(precision):
    """rmpcd_md_substep: the interval's n_md velocity-Verlet sub-steps run one
    call at a time equal rmpcd_stream's whole interval bit for bit (solvent,
    species, colloids), the RATTLE bond holds after every sub-step, and the
    sub-steps must come in order."""
    cfg, col, bonds, x, v, fl = _dimer(precision)
    col[0]["v"] = (0.03, -0.01, 0.0)
    col[1]["v"] = (0.03, -0.01, 0.0)
    a = gpu(cfg, x, v, fl, col, bonds, precision=precision, step=3)
    a.stream_interval()
    sa, ca = a.get_state(), a.get_colloids(0)
    b = gpu(cfg, x, v, fl, col, bonds, precision=precision, step=3)
    with pytest.raises(api.RmpcdError) as e:
        b.md_substep(1)
    assert e.value.code == "ESTATE"
    prev = b.get_colloids(0)["x"]
    moved = 0
    for k in range(cfg["n_md"]):
        b.md_substep(k)
        if k < cfg["n_md"] - 1:
            X = b.get_colloids(0)["x"]
            bond = np.linalg.norm(X[0] - X[1])
            assert abs(bond - 4.5) < (1e-11 if precision == "fp64" else 1e-5), (k, bond)
            moved += np.abs(X - prev).max() > 0
            prev = X
            if k == 5:
                with pytest.raises(api.RmpcdError) as e:
                    b.get_state()
                assert e.value.code == "ESTATE"
    assert moved >= cfg["n_md"] - 2
    sb, cb2 = b.get_state(), b.get_colloids(0)
    for key in ("id", "x", "v", "flags"):
        assert np.array_equal(sa[key], sb[key]), key
    assert np.array_equal(ca["x"], cb2["x"]) and np.array_equal(ca["v"], cb2["v"])
    # the interval is closed: the next step runs
    b.step(1)
    b.sync()
