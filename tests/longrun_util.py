"""Long-run observables of replica ensembles of the reactive sphere dimer, on
the GPU path (mixed or FP64) and on the oracle: the solvent temperature, the
solvent self-diffusion coefficient and the dimer's directed speed, each as a
per-replica mean so that the spread across independent replicas gives the
standard error.

Definitions (the same on every side):
  T  -- the cell-frame temperature of §1.4 (cells with N >= 2), averaged over
        samples taken every t_every intervals of the run;
  D  -- from the solvent's mean squared displacement in windows: snapshots at
        t0, t0 + a and t0 + b intervals (minimum-image displacements, which
        hold while b tau stays short against half the box),
        D = (MSD(b) - MSD(a)) / (6 (b - a) tau), the difference removing the
        ballistic offset of the first collisions; averaged over windows;
  V  -- the dimer's directed speed: displacement of its centre of mass over
        w intervals projected on its axis u = (X_N - X_C) / |X_N - X_C| at the
        window start, divided by w tau; averaged over windows.
"""
import math

import numpy as np

from paper_1608_04904_gb300 import synth


def dimer_replica(r, L=16):
    cfg, col, bonds = synth.dimer32(precision="mixed", seed=2 + r, L=L)
    x, v, fl = synth.solvent(cfg, col, seed=1000 + r)
    return cfg, col, bonds, (x, v, fl)


def _min_image(d, L):
    L = np.asarray(L, float)
    return d - L * np.round(d / L)


class _Acc:
    """Samples per replica as (interval index of the window end, value)."""

    def __init__(self, R):
        self.T = [[] for _ in range(R)]
        self.D = [[] for _ in range(R)]
        self.V = [[] for _ in range(R)]

    def result(self):
        return {"T": self.T, "D": self.D, "V": self.V}


def per_replica(samples, k_max=None):
    """Per-replica means of the samples whose window ends at or before k_max
    (all samples when None): equal time windows on every side, since the
    reactions heat the unthermostatted dimer system slowly."""
    return np.array([np.mean([v for k, v in s if k_max is None or k <= k_max]) for s in samples])


def _schedule(K, a, b, n_win, w):
    """Intervals (from the start of production) at which each window starts."""
    d_starts = [int(k * K / n_win) for k in range(n_win)]
    assert d_starts[-1] + b <= K
    v_starts = list(range(0, K - w + 1, w))
    return d_starts, v_starts


def run_gpu(api, precision, R, warm, K, t_every=50, a=2, b=8, n_win=10, w=20, L=16):
    """R dimer replicas in one batched system, warm + K fused intervals."""
    reps = [dimer_replica(r, L) for r in range(R)]
    s = api.System([dict(cfg=c, n=len(st[0]), colloids=col, bonds=bo) for c, col, bo, st in reps],
                   precision=precision, bucket_cap=0)
    for r, (_, _, _, (x, v, fl)) in enumerate(reps):
        s.set_state(r, x, v, fl)
    s.step(warm)
    tau = reps[0][0]["tau"]
    Lb = reps[0][0]["L"]
    acc = _Acc(R)
    d_starts, v_starts = _schedule(K, a, b, n_win, w)
    snaps = {}
    vstart = {}
    for k in range(K + 1):
        if k % t_every == 0 and k > 0:
            for r in range(R):
                acc.T[r].append((k, s.observables(r)["temperature"]))
        for j, t0 in enumerate(d_starts):
            if k in (t0, t0 + a, t0 + b):
                for r in range(R):
                    st = s.get_state(r)
                    o = np.argsort(st["id"])
                    snaps[(j, k - t0, r)] = st["x"][o]
                if k == t0 + b:
                    for r in range(R):
                        x0 = snaps.pop((j, 0, r))
                        da = _min_image(snaps.pop((j, a, r)) - x0, Lb)
                        db = _min_image(snaps.pop((j, b, r)) - x0, Lb)
                        msd_a = float((da * da).sum(1).mean())
                        msd_b = float((db * db).sum(1).mean())
                        acc.D[r].append((k, (msd_b - msd_a) / (6.0 * (b - a) * tau)))
        if k in vstart or k in v_starts:
            for r in range(R):
                X = s.get_colloids(r)["x"]
                if k in vstart:
                    X0, u = vstart[k][r]
                    acc.V[r].append((k, float(np.dot(X.mean(0) - X0, u)) / (w * tau)))
                if k in v_starts and k + w <= K:
                    ax = X[1] - X[0]
                    vstart.setdefault(k + w, {})[r] = (X.mean(0), ax / np.linalg.norm(ax))
            vstart.pop(k, None)
        if k < K:
            s.step(1)
    s.close()
    return acc.result()


def run_oracle(orc, R, warm, K, t_every=50, a=2, b=8, n_win=10, w=20, L=16):
    """The same measurement on the oracle, replica by replica."""
    acc = _Acc(R)
    d_starts, v_starts = _schedule(K, a, b, n_win, w)
    for r in range(R):
        cfg, col, bonds, (x, v, fl) = dimer_replica(r, L)
        o = orc.OracleSystem(cfg, x, v, fl, colloids=synth.colloid_arrays(col), bonds=bonds)
        o.step(warm)
        tau, Lb = cfg["tau"], cfg["L"]
        snap = {}
        vst = {}
        for k in range(K + 1):
            if k % t_every == 0 and k > 0:
                acc.T[r].append((k, o.temperature()))
            for j, t0 in enumerate(d_starts):
                if k in (t0, t0 + a, t0 + b):
                    snap[(j, k - t0)] = o.x[np.argsort(o.id)].copy()
                if k == t0 + b:
                    x0 = snap.pop((j, 0))
                    da = _min_image(snap.pop((j, a)) - x0, Lb)
                    db = _min_image(snap.pop((j, b)) - x0, Lb)
                    acc.D[r].append((k, (float((db * db).sum(1).mean()) - float((da * da).sum(1).mean()))
                                     / (6.0 * (b - a) * tau)))
            if k in vst:
                X0, u = vst.pop(k)
                acc.V[r].append((k, float(np.dot(o.X.mean(0) - X0, u)) / (w * tau)))
            if k in v_starts and k + w <= K:
                ax = o.X[1] - o.X[0]
                vst[k + w] = (o.X.mean(0).copy(), ax / np.linalg.norm(ax))
            if k < K:
                o.step(1)
    return acc.result()


def mean_se(a):
    a = np.asarray(a, float)
    return float(a.mean()), float(a.std(ddof=1) / math.sqrt(len(a)))


def compare(name, got, ref, rel=0.01, nse=3.0, need_rel=True):
    """Pass iff |mean_got - mean_ref| <= nse * sqrt(SE_got^2 + SE_ref^2) and,
    with need_rel, also <= rel * |mean_ref|.  Returns the record."""
    mg, sg = mean_se(got)
    mr, sr = mean_se(ref)
    d = mg - mr
    se = math.sqrt(sg * sg + sr * sr)
    rec = {"obs": name, "got": mg, "se_got": sg, "ref": mr, "se_ref": sr, "diff": d,
           "rel": d / mr if mr else float("nan"), "z": d / se if se > 0 else float("inf"),
           "rel_se": se / abs(mr) if mr else float("nan")}
    ok = abs(d) <= nse * se and (not need_rel or abs(d) <= rel * abs(mr))
    return ok, rec
