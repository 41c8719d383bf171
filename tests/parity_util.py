"""Helpers of the GPU-vs-oracle parity tests.

Tolerances (per velocity component, relative to max(|v_oracle|, sqrt(kT))):
  fp64 path 1e-12, mixed path 1e-5.  Positions: absolute 1e-12 * L (fp64) and
  1e-5 (mixed, cell side 1), compared modulo the box on periodic axes.  The
  mixed path's few exceptions are bounded by check_mixed_exceptions.
"""
import numpy as np

TOL = {"fp64": 1e-12, "mixed": 1e-5}


def vel_bad(v_gpu, v_orc, kT, precision):
    scale = np.maximum(np.abs(v_orc), np.sqrt(kT) if kT > 0 else 1.0)
    return (np.abs(v_gpu - v_orc) > TOL[precision] * scale).any(axis=1)


def pos_diff(x_gpu, x_orc, L, walls):
    """x_gpu - x_orc, taken modulo the box on the periodic axes."""
    L = np.asarray(L, float)
    d = x_gpu - x_orc
    per = np.ones(3, bool)
    if walls:
        per[2] = False
    d[:, per] -= L[per] * np.round(d[:, per] / L[per])
    return d


def pos_bad(x_gpu, x_orc, L, walls, precision):
    L = np.asarray(L, float)
    d = pos_diff(x_gpu, x_orc, L, walls)
    tol = TOL[precision] * (L.max() if precision == "fp64" else 1.0)
    return (np.abs(d) > tol).any(axis=1)


def check_mixed_exceptions(bad, near, flag_diff, dv, kT, allow, what="velocity"):
    """The mixed path's exceptions to its 1e-5 tolerance, bounded.

    FP32 arithmetic can put a particle on the other side of a threshold that
    the FP64 oracle decides: a cut-off of the WCA force or a catalytic range,
    both met only by particles that spend the interval near a colloid (the
    oracle's near flag), and a tagged particle whose conversion then differs
    (its species flag).  So a particle beyond the tolerance must be near or
    have a differing flag, there may be at most `allow` of them, and each
    stays within the thermal scale (|dv| < sqrt(kT)) -- a wrong term in the
    arithmetic shows up everywhere, or far above that."""
    bad = np.asarray(bad, bool)
    idx = np.flatnonzero(bad)
    info = [(int(i), bool(near[i]), bool(flag_diff[i]), float(np.abs(dv[i]).max())) for i in idx[:8]]
    assert len(idx) <= allow, (what, len(idx), info)
    assert np.all(near[idx] | flag_diff[idx]), (what, "exception away from every colloid", info)
    assert np.all(np.abs(dv[idx]) < np.sqrt(kT)), (what, "exception beyond the thermal scale", info)
    return info


def by_id(state_ids, *arrays):
    order = np.argsort(state_ids)
    return [a[order] for a in arrays]


def near_boundary(x, s, eps):
    """Particles whose position lies within eps of a plane of the shifted grid."""
    f = x - s
    frac = f - np.floor(f)
    return ((frac < eps) | (frac > 1.0 - eps)).any(axis=1)


def compare_step(cfg, st, o, precision):
    """Compare a GPU state with the oracle's after full intervals."""
    gid, gx, gv, gf, gc = by_id(st["id"], st["id"], st["x"], st["v"], st["flags"], st["cell"])
    oid, ox, ov, of, oc, onear = by_id(o.id, o.id, o.x, o.v, o.flags, o.key, o.near.astype(bool))
    assert np.array_equal(gid, oid)
    if precision == "fp64":
        assert np.array_equal(st["id"], o.id)
        assert np.array_equal(gc, oc)
        assert np.array_equal(gf, of)
        assert not pos_bad(gx, ox, cfg["L"], cfg.get("walls", 0), "fp64").any()
        assert not vel_bad(gv, ov, cfg["kT"], "fp64").any()
        return
    # mixed: keys may differ for particles that FP32 flight puts on the other
    # side of a cell plane; those cells are excluded from the velocity check
    mism = gc != oc
    s = o.shift
    border = near_boundary(ox, s, 1e-4)
    assert np.all(border[mism]), "key mismatch away from a cell boundary"
    assert mism.sum() <= max(3, 1e-4 * len(gc))
    badcells = np.isin(oc, oc[mism]) | np.isin(oc, gc[mism])
    assert not pos_bad(gx, ox, cfg["L"], cfg.get("walls", 0), "mixed").any()
    vb = vel_bad(gv, ov, cfg["kT"], "mixed") & ~badcells
    check_mixed_exceptions(vb, onear, gf != of, gv - ov, cfg["kT"], 2)
    assert (gf != of).sum() <= 2 + mism.sum()
