"""Seeded synthetic systems shaped like the paper's simulation setups.

This module only builds inputs: parameter dicts and initial solvent/colloid
states drawn with numpy's PCG64.  It holds none of the method's arithmetic and
is shared by the tests, ``bench.py`` and the oracle checks.

Positions are drawn as integer multiples of 2^-24 so that ``cell + offset``
with an FP32 offset represents them exactly; for the mixed-precision path the
velocities are rounded to FP32 values, so both sides of a parity test start
from the same numbers.

Workloads (stand-ins for the paper's ``experiments/``, §1.5 and Appendix A):

* ``sphere16``   -- 16^3 periodic box, rho = 10, one WCA sphere (sigma 2, M 200),
  alpha 130 deg, tau 0.5, 50 MD sub-steps, FP64.
* ``dimer32``    -- reactive sphere-dimer nanomotor (``single_dimer_pbc``), 32^3,
  rho = 10, catalytic C and inert N (sigma 2, M 100, bond 4.5), kT = 1/3,
  alpha 90 deg, tau 0.5, 50 sub-steps, A->B on leaving C, bulk B->A k = 0.01.
* ``poiseuille128`` -- 128^3 channel with stick walls at z = 0, 128, body
  acceleration 0.001 along x, alpha 130 deg, tau 1 (``poiseuille_flow``).
* ``thermal256`` -- 256 x 64 x 64, 64 WCA spheres (sigma 2.5, M 150), MPC-AT
  slabs at kT 1.2 / 0.8, colloid-colloid LJ (``single_sphere_thermo_trap``).
* ``batch``      -- independent replicas with cubic sides drawn from
  {16, 20, 24, 32, 40, 48}, each holding one Janus particle built from 100-300
  beads on a sphere of radius 4 (``single_janus_pbc``).
"""
from __future__ import annotations

import math

import numpy as np

WCA_RC_FACTOR = 2.0 ** (1.0 / 6.0)


def base_config(**kw) -> dict:
    cfg = {
        "L": (16, 16, 16), "rho": 10, "kT": 1.0, "alpha": math.radians(130.0), "tau": 0.5,
        "n_md": 50, "walls": 0, "rho_wall": 0, "g": (0.0, 0.0, 0.0), "bulk_rate": 0.0,
        "cat_prob": 1.0, "skin": 0.5, "slabs": [], "cc_lj": None, "seed": 1,
        "precision": "fp64", "bucket_cap": 0,
    }
    cfg.update(kw)
    return cfg


def sphere16(precision="fp64", seed=1):
    cfg = base_config(L=(16, 16, 16), alpha=math.radians(130.0), tau=0.5, n_md=50, kT=1.0,
                      seed=seed, precision=precision)
    col = [dict(x=(8.0, 8.0, 8.0), v=(0.0, 0.0, 0.0), mass=200.0, sigma=2.0, eps_A=1.0, eps_B=1.0,
                catalytic=0)]
    return cfg, col, []


def dimer32(precision="mixed", seed=2, L=32):
    cfg = base_config(L=(L, L, L), alpha=math.radians(90.0), tau=0.5, n_md=50, kT=1.0 / 3.0,
                      bulk_rate=0.01, cat_prob=1.0, seed=seed, precision=precision)
    c = L / 2.0
    col = [dict(x=(c - 2.25, c, c), v=(0.0, 0.0, 0.0), mass=100.0, sigma=2.0, eps_A=1.0, eps_B=1.0,
                catalytic=1),
           dict(x=(c + 2.25, c, c), v=(0.0, 0.0, 0.0), mass=100.0, sigma=2.0, eps_A=1.0, eps_B=0.1,
                catalytic=0)]
    return cfg, col, [(0, 1, 4.5)]


def poiseuille(precision="mixed", seed=3, L=(128, 128, 128), g=0.001):
    cfg = base_config(L=tuple(L), alpha=math.radians(130.0), tau=1.0, n_md=1, kT=1.0, walls=1,
                      rho_wall=10, g=(g, 0.0, 0.0), seed=seed, precision=precision)
    return cfg, [], []


def thermal(precision="mixed", seed=5, L=(256, 64, 64), n_spheres=64):
    cfg = base_config(L=tuple(L), alpha=math.radians(130.0), tau=0.5, n_md=50, kT=1.0,
                      slabs=[(0.0, 8.0, 1.2), (L[0] / 2.0, L[0] / 2.0 + 8.0, 0.8)],
                      cc_lj=(1.0, 5.5, 2.5 * 5.5), seed=seed, precision=precision)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    pos = []
    dmin = WCA_RC_FACTOR * 5.5
    while len(pos) < n_spheres:
        p = rng.uniform(0, 1, 3) * np.asarray(L, float)
        ok = True
        for q in pos:
            d = p - q
            d -= np.asarray(L) * np.round(d / np.asarray(L))
            if np.dot(d, d) < dmin * dmin:
                ok = False
                break
        if ok:
            pos.append(p)
    col = [dict(x=tuple(p), v=(0.0, 0.0, 0.0), mass=150.0, sigma=2.5, eps_A=1.0, eps_B=1.0, catalytic=0)
           for p in pos]
    return cfg, col, []


def colloid_arrays(col) -> dict:
    n = len(col)
    return {
        "x": np.asarray([c["x"] for c in col], dtype=np.float64).reshape(n, 3),
        "v": np.asarray([c["v"] for c in col], dtype=np.float64).reshape(n, 3),
        "mass": np.asarray([c["mass"] for c in col], dtype=np.float64),
        "sigma": np.asarray([c["sigma"] for c in col], dtype=np.float64),
        "eps_A": np.asarray([c["eps_A"] for c in col], dtype=np.float64),
        "eps_B": np.asarray([c["eps_B"] for c in col], dtype=np.float64),
        "catalytic": np.asarray([c["catalytic"] for c in col], dtype=np.int32),
    }


def _inside_any(x, centers, radii, L):
    """Mask of the points x that lie within radius of any centre (minimum
    image), testing only the points in the cells around each centre."""
    bad = np.zeros(len(x), dtype=bool)
    if len(centers) == 0 or len(x) == 0:
        return bad
    cells = np.floor(x).astype(np.int64) % L
    key = cells[:, 0] + L[0] * (cells[:, 1] + L[1] * cells[:, 2])
    order = np.argsort(key, kind="stable")
    skey = key[order]
    for c, r in zip(centers, radii):
        c = np.mod(c, L)
        lo = np.floor(c - r).astype(np.int64)
        hi = np.floor(c + r).astype(np.int64)
        rng_ = [np.arange(lo[d], hi[d] + 1) % L[d] for d in range(3)]
        cz, cy, cx_ = np.meshgrid(rng_[2], rng_[1], rng_[0], indexing="ij")
        want = np.unique((cx_ + L[0] * (cy + L[1] * cz)).ravel())
        a = np.searchsorted(skey, want, side="left")
        b = np.searchsorted(skey, want, side="right")
        idx = np.concatenate([order[i:j] for i, j in zip(a, b)]) if len(want) else np.zeros(0, np.int64)
        if len(idx) == 0:
            continue
        d = x[idx] - c
        d -= L * np.round(d / L)
        bad[idx[(d * d).sum(1) < r * r]] = True
    return bad


def solvent(cfg, col=(), n=None, seed=None, frac_b=0.0, tag_frac=0.0, exclude=True, exclude_factor=None):
    """Uniform positions (multiples of 2^-24) outside every colloid's cut-off
    (or outside ``exclude_factor * sigma`` when given),
    Maxwell-Boltzmann velocities at kT with the mean removed, species A (or a
    fraction ``frac_b`` of B)."""
    L = np.asarray(cfg["L"], dtype=np.int64)
    if n is None:
        n = int(cfg["rho"] * L.prod())
    rng = np.random.Generator(np.random.PCG64(cfg["seed"] if seed is None else seed))
    scale = np.int64(1) << np.int64(24)
    x = np.empty((n, 3), dtype=np.float64)
    todo = np.arange(n)
    cx = np.asarray([c["x"] for c in col], dtype=np.float64).reshape(-1, 3)
    fac = WCA_RC_FACTOR if exclude_factor is None else exclude_factor
    rcs = np.asarray([fac * c["sigma"] for c in col], dtype=np.float64)
    for _ in range(1000):
        k = len(todo)
        if k == 0:
            break
        ints = rng.integers(0, L * scale, size=(k, 3), dtype=np.int64)
        x[todo] = ints.astype(np.float64) * 2.0 ** -24
        if not exclude or len(col) == 0:
            todo = todo[:0]
            break
        bad = _inside_any(x[todo], cx, rcs, L)
        todo = todo[bad]
    v = rng.standard_normal((n, 3)) * math.sqrt(cfg["kT"])
    if n > 0:
        v -= v.mean(axis=0)
    if cfg.get("precision", "fp64") == "mixed":
        v = v.astype(np.float32).astype(np.float64)
    flags = np.zeros(n, dtype=np.uint8)
    if frac_b > 0:
        flags |= (rng.uniform(size=n) < frac_b).astype(np.uint8)
    if tag_frac > 0:
        flags |= ((rng.uniform(size=n) < tag_frac) & ((flags & 1) == 0)).astype(np.uint8) * 2
    return x, v, flags


def batch_sides(n_replicas, seed=4):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(s) for s in rng.choice([16, 20, 24, 32, 40, 48], size=n_replicas)]


def batch_sphere(side, seed, precision="mixed"):
    """One replica of the batched ensemble: a cube of the given side at
    density 10 holding one WCA sphere of radius 4 (sigma 4) at the centre with
    the mass of the displaced solvent (neutral buoyancy), alpha 130 deg,
    tau 0.5, 25 MD sub-steps of dt 0.02.  The sphere stands in for the
    bead-built Janus particle of the same radius."""
    L = (side, side, side)
    cfg = base_config(L=L, alpha=math.radians(130.0), tau=0.5, n_md=25, kT=1.0, seed=seed, precision=precision)
    m = 10.0 * 4.0 / 3.0 * math.pi * 4.0 ** 3
    c = side / 2.0
    col = [dict(x=(c, c, c), v=(0.0, 0.0, 0.0), mass=m, sigma=4.0, eps_A=1.0, eps_B=1.0, catalytic=1)]
    return cfg, col, []


def fibonacci_sphere(nb: int, radius: float) -> np.ndarray:
    """nb nearly uniform points on a sphere (Fibonacci lattice): heights
    z_j = 1 - (2 j + 1) / nb, azimuths j times the golden angle."""
    j = np.arange(nb, dtype=np.float64)
    z = 1.0 - (2.0 * j + 1.0) / nb
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = j * (math.pi * (3.0 - math.sqrt(5.0)))
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def bead_links(x, factor: float = 1.35):
    """Links of a bead network for the iterative-RATTLE model of the Janus
    particle: every bead pair closer than `factor` times the median
    nearest-neighbour distance (on a Fibonacci shell this joins each bead to
    its ring of neighbours).  Returns (pairs, lengths)."""
    x = np.asarray(x, dtype=np.float64)
    dist = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(dist, np.inf)
    cut = factor * float(np.median(dist.min(1)))
    a, b = np.nonzero(np.triu(dist < cut, 1))
    return [(int(i), int(j)) for i, j in zip(a, b)], dist[a, b]


def matrix_quaternion(R) -> np.ndarray:
    """Unit quaternion (w, x, y, z) of a proper rotation matrix (Shepperd's
    branch on the largest diagonal term)."""
    R = np.asarray(R, dtype=np.float64)
    t = np.trace(R)
    if t > 0:
        s = 2.0 * math.sqrt(1.0 + t)
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    else:
        i = int(np.argmax(np.diag(R)))
        j, k = (i + 1) % 3, (i + 2) % 3
        s = 2.0 * math.sqrt(1.0 + R[i, i] - R[j, j] - R[k, k])
        q = [0.0] * 4
        q[0] = (R[k, j] - R[j, k]) / s
        q[1 + i] = 0.25 * s
        q[1 + j] = (R[j, i] + R[i, j]) / s
        q[1 + k] = (R[k, i] + R[i, k]) / s
    q = np.asarray(q)
    return q / np.linalg.norm(q)


def janus_body(nb: int, center, seed: int, radius: float = 4.0, rho: float = 10.0, sigma: float = 1.0,
               eps_A=1.0, eps_B=1.0, kT: float = 1.0, thermal: bool = True) -> dict:
    """A Janus particle of nb beads on a Fibonacci sphere of the given radius,
    catalytic where the construction frame has z > 0, with equal bead masses
    totalling rho (4/3) pi radius^3 (neutral buoyancy).  The beads are centred
    and expressed in the principal frame of their inertia tensor; the
    orientation q maps that frame back onto the construction frame.  With
    ``thermal`` the centre-of-mass velocity and body-frame angular momentum
    are drawn from Maxwell-Boltzmann at kT, else both are zero."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    b0 = fibonacci_sphere(nb, radius)
    cat = (b0[:, 2] > 0.0).astype(np.int32)
    b0 = b0 - b0.mean(axis=0)
    m_b = rho * 4.0 / 3.0 * math.pi * radius ** 3 / nb
    It = m_b * ((b0 * b0).sum() * np.eye(3) - b0.T @ b0)
    w, E = np.linalg.eigh(It)
    if np.linalg.det(E) < 0:
        E[:, 2] = -E[:, 2]
    b = b0 @ E                        # b0 = E b  (rows: b = E^T b0)
    q = matrix_quaternion(E)
    M = m_b * nb
    Ib = m_b * np.array([(b[:, 1] ** 2 + b[:, 2] ** 2).sum(), (b[:, 2] ** 2 + b[:, 0] ** 2).sum(),
                         (b[:, 0] ** 2 + b[:, 1] ** 2).sum()])
    if thermal:
        v = rng.standard_normal(3) * math.sqrt(kT / M)
        l = rng.standard_normal(3) * np.sqrt(kT * Ib)
    else:
        v = np.zeros(3)
        l = np.zeros(3)
    return {"x": np.asarray(center, dtype=np.float64), "v": v, "q": q, "l": l, "b": b,
            "eps_A": np.broadcast_to(np.asarray(eps_A, np.float64), nb).copy(),
            "eps_B": np.broadcast_to(np.asarray(eps_B, np.float64), nb).copy(),
            "catalytic": cat, "bead_mass": m_b, "sigma": sigma}


def janus_network(body, radius: float = 4.0, factor: float = 1.6) -> dict:
    """The beads of a Janus body description (``janus_body`` of the same
    radius) as a bead network for iterative RATTLE: positions on the
    construction-frame sphere about the body's centre, every bead moving with
    the body's centre-of-mass velocity (a rigid translation, so the links hold
    and their velocities agree from the start), the body's masses,
    couplings and catalytic flags, and links joining every bead pair closer
    than `factor` times the median nearest-neighbour distance (``bead_links``).
    At 1.6 a shell of 100-300 beads has more than 3 nb - 6 links, so the
    network is rigid; the sparser ring-of-neighbours network (1.35) leaves
    floppy modes, along which the iterative RATTLE can need more than 10^4
    sweeps."""
    nb = len(body["b"])
    b0 = fibonacci_sphere(nb, radius)
    b0 = b0 - b0.mean(axis=0)
    links, d = bead_links(b0, factor=factor)
    return {"xb": np.asarray(body["x"], np.float64) + b0,
            "vb": np.broadcast_to(np.asarray(body["v"], np.float64), (nb, 3)).copy(),
            "mb": np.full(nb, float(body["bead_mass"])), "eps_A": np.asarray(body["eps_A"], np.float64),
            "eps_B": np.asarray(body["eps_B"], np.float64), "catalytic": np.asarray(body["catalytic"], np.int32),
            "sigma": float(body["sigma"]), "links": links, "d": np.asarray(d, np.float64)}


def body_exclusion(body) -> list:
    """A pseudo-colloid whose cut-off covers the body's bounding sphere, for
    ``solvent(..., col=...)``: no solvent starts inside the bead shell."""
    b = np.asarray(body["b"])
    reach = float(np.sqrt((b * b).sum(1)).max()) + WCA_RC_FACTOR * body["sigma"]
    return [dict(x=tuple(body["x"]), sigma=reach / WCA_RC_FACTOR)]


def batch_janus(side, seed, precision="mixed", nb=None):
    """One replica of the batched ensemble: a cube of the given side at
    density 10 holding one Janus particle of nb beads (drawn from
    U{100..300} with the replica's seed when not given) on a sphere of radius 4
    at the centre, sigma_b = 1, eps = 1, catalytic hemisphere (A -> B with
    probability 1), alpha 130 deg, tau 0.5, 25 MD sub-steps of dt 0.02."""
    L = (side, side, side)
    cfg = base_config(L=L, alpha=math.radians(130.0), tau=0.5, n_md=25, kT=1.0, seed=seed, precision=precision)
    if nb is None:
        nb = int(np.random.Generator(np.random.PCG64(seed + 104729)).integers(100, 301))
    c = side / 2.0
    body = janus_body(nb, (c, c, c), seed)
    return cfg, body
