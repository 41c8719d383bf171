"""FP64 CPU oracle of one MPCD collision interval -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this module.  The product package never imports it,
and it imports nothing from the product package: the oracle and the CUDA path
share no code.  The arithmetic lives in ``rmpcd_oracle.c`` (compiled here with
gcc, ``-ffp-contract=off``); this file only marshals numpy arrays.

Order of one collision interval (the paper lists the ingredients in §1.4 but
not their order; this is the reading used throughout):

    interval motion (MD sub-steps near colloids, free flight elsewhere)
    -> random grid shift -> stable sort into cells -> collision (SRD / MPC-AT /
    virtual wall particles) -> bulk B->A reaction -> step counter + 1
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmpcd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

F_B = 1      # species B
F_TAG = 2    # A particle inside a catalytic colloid's range


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-Wall", "-Wextra", "-Wno-unused-parameter",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("L", C.c_int32 * 3), ("walls", C.c_int32), ("rho_wall", C.c_int32),
        ("n_md", C.c_int32), ("n_slabs", C.c_int32), ("bulk_mode", C.c_int32),
        ("kT", C.c_double), ("alpha", C.c_double), ("tau", C.c_double),
        ("g", C.c_double * 3), ("bulk_rate", C.c_double), ("cat_prob", C.c_double),
        ("skin", C.c_double),
        ("slab_x0", C.c_double * 4), ("slab_x1", C.c_double * 4), ("slab_kT", C.c_double * 4),
        ("cc_eps", C.c_double), ("cc_sigma", C.c_double), ("cc_rc", C.c_double),
        ("seed", C.c_uint64),
    ]


def make_params(cfg: dict) -> Params:
    """Fill the oracle's parameter struct from a plain configuration dict."""
    p = Params()
    p.L[:] = [int(a) for a in cfg["L"]]
    p.walls = int(cfg.get("walls", 0))
    p.rho_wall = int(cfg.get("rho_wall", 0))
    p.n_md = int(cfg.get("n_md", 1))
    slabs = cfg.get("slabs", [])
    p.n_slabs = len(slabs)
    for k, (x0, x1, kt) in enumerate(slabs):
        p.slab_x0[k], p.slab_x1[k], p.slab_kT[k] = x0, x1, kt
    p.bulk_mode = 1 if cfg.get("bulk_rate", 0.0) > 0.0 else 0
    p.kT = float(cfg["kT"])
    p.alpha = float(cfg["alpha"])
    p.tau = float(cfg["tau"])
    p.g[:] = [float(a) for a in cfg.get("g", (0.0, 0.0, 0.0))]
    p.bulk_rate = float(cfg.get("bulk_rate", 0.0))
    p.cat_prob = float(cfg.get("cat_prob", 1.0))
    p.skin = float(cfg.get("skin", 0.5))
    cc = cfg.get("cc_lj")
    if cc:
        p.cc_eps, p.cc_sigma, p.cc_rc = cc
    p.seed = int(cfg["seed"]) & 0xFFFFFFFFFFFFFFFF
    return p


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's per-particle and per-cell loops (0 = every
    core of the host); returns the count in use.  Results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i64, u32, u8, i32 = C.c_double, C.c_int64, C.c_uint32, C.c_uint8, C.c_int32
            P = C.POINTER
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            L.orc_get_threads.restype = C.c_int
            L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            L.orc_grid_shift.argtypes = [C.c_uint64, u32, P(d)]
            L.orc_rotation_axis.argtypes = [C.c_uint64, u32, u32, P(d)]
            L.orc_n_cells.argtypes = [P(Params)]
            L.orc_n_cells.restype = i64
            L.orc_cell_keys.argtypes = [P(Params), i64, P(d), P(d), P(i32)]
            L.orc_counting_sort.argtypes = [i64, P(i32), P(u32), i64, P(i64), P(i64), P(i64)]
            L.orc_gather.argtypes = [i64, P(i64), C.c_void_p, C.c_void_p, i64]
            L.orc_collide.argtypes = [P(Params), u32, i64, P(i64), P(i64), P(d)]
            L.orc_bulk_react.argtypes = [P(Params), u32, i64, P(i64), P(i64), P(u8)]
            L.orc_flight.argtypes = [P(Params), i64, P(d), P(d), P(u8)]
            L.orc_wca_force.argtypes = [P(d), d, d, d, P(d), P(d)]
            L.orc_wca_force.restype = C.c_int
            L.orc_wca_rc2.argtypes = [d]
            L.orc_wca_rc2.restype = d
            L.orc_interval.argtypes = [P(Params), u32, i64, P(d), P(d), P(u8), P(u32),
                                       C.c_int, P(d), P(d), P(d), P(d), P(d), P(d), P(i32),
                                       C.c_int, P(i32), P(i32), P(d), C.c_int, P(u8)]
            L.orc_interval.restype = C.c_int
            L.orc_forces.argtypes = [P(Params), i64, P(d), P(u8), C.c_int, P(d), P(d), P(d), P(d),
                                     P(d), P(d)]
            L.orc_potential_energy.argtypes = [P(Params), i64, P(d), P(u8), C.c_int, P(d), P(d), P(d), P(d),
                                               C.c_int, P(i32), P(i32)]
            L.orc_potential_energy.restype = d
            L.orc_temperature.argtypes = [i64, P(i64), P(i64), P(d), P(i64)]
            L.orc_temperature.restype = d
            L.orc_quat_matrix.argtypes = [P(d), P(d)]
            L.orc_body_inertia.argtypes = [C.c_int, P(d), d, P(d), P(d)]
            L.orc_body_reach.argtypes = [C.c_int, P(d), d]
            L.orc_body_reach.restype = d
            L.orc_body_rotate.argtypes = [P(d), d, P(d), P(d)]
            L.orc_interval_body.argtypes = [P(Params), u32, i64, P(d), P(d), P(u8), P(u32),
                                            C.c_int, P(d), P(d), P(d), P(i32), d, d,
                                            P(d), P(d), P(d), P(d), C.c_int, P(u8)]
            L.orc_interval_body.restype = C.c_int
            L.orc_body_forces.argtypes = [P(Params), i64, P(d), P(u8), C.c_int, P(d), P(d), P(d), P(i32),
                                          d, P(d), P(d), P(d), P(d), P(d)]
            L.orc_body_forces.restype = d
            L.orc_rattle_pos_iter.argtypes = [C.c_int, P(i32), P(i32), P(d), P(d), P(d), P(d), P(d), d, d, C.c_int]
            L.orc_rattle_pos_iter.restype = C.c_int
            L.orc_rattle_vel_iter.argtypes = [C.c_int, P(i32), P(i32), P(d), P(d), P(d), P(d), d, C.c_int]
            L.orc_rattle_vel_iter.restype = C.c_int
            L.orc_network_step.argtypes = [C.c_int, P(d), C.c_int, P(i32), P(i32), P(d), P(d), P(d), P(d), d, d,
                                           C.c_int]
            L.orc_network_step.restype = C.c_int
            L.orc_interval_network.argtypes = [P(Params), u32, i64, P(d), P(d), P(u8), P(u32), C.c_int, P(d), P(d),
                                               P(d), P(d), P(d), P(i32), d, C.c_int, P(i32), P(i32), P(d), d,
                                               C.c_int, C.c_int, P(u8)]
            L.orc_interval_network.restype = C.c_int
            L.orc_network_energy.argtypes = [P(Params), i64, P(d), P(u8), C.c_int, P(d), P(d), P(d), P(i32), d]
            L.orc_network_energy.restype = d
            L.orc_hilbert_index.argtypes = [C.c_int, u32, u32, u32]
            L.orc_hilbert_index.restype = C.c_uint64
            L.orc_hilbert_rank.argtypes = [P(i32), P(i64)]
            L.orc_hilbert_rank.restype = C.c_int
            L.orc_species_reservoirs.argtypes = [P(Params), i64, P(i64), P(i64), P(u8), i32, i32, i32, i32]
            L.orc_species_reservoirs.restype = None
            L.orc_cc_forces.argtypes = [P(Params), C.c_int, P(d), C.c_int, P(i32), P(i32), P(d)]
            L.orc_cc_forces.restype = None
            _lib = L
    return _lib


# --------------------------------------------------------------------------
# thin functional wrappers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def grid_shift(seed: int, step: int) -> np.ndarray:
    s = np.zeros(3)
    lib().orc_grid_shift(C.c_uint64(seed), step, _ptr(s, C.c_double))
    return s


def rotation_axis(seed: int, step: int, cell: int) -> np.ndarray:
    n = np.zeros(3)
    lib().orc_rotation_axis(C.c_uint64(seed), step, cell, _ptr(n, C.c_double))
    return n


def wca_force(d, sigma, eps, rc2=None):
    d = np.ascontiguousarray(d, dtype=np.float64)
    f = np.zeros(3)
    e = np.zeros(1)
    if rc2 is None:
        rc2 = lib().orc_wca_rc2(sigma)
    hit = lib().orc_wca_force(_ptr(d, C.c_double), sigma, eps, rc2, _ptr(f, C.c_double), _ptr(e, C.c_double))
    return bool(hit), f, float(e[0])


def n_cells(cfg) -> int:
    p = make_params(cfg)
    return int(lib().orc_n_cells(C.byref(p)))


def cell_keys(cfg, x, s) -> np.ndarray:
    p = make_params(cfg)
    x = np.ascontiguousarray(x, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    key = np.zeros(len(x), dtype=np.int32)
    lib().orc_cell_keys(C.byref(p), len(x), _ptr(x, C.c_double), _ptr(s, C.c_double), _ptr(key, C.c_int32))
    return key


def counting_sort(key, ncells, ids=None):
    """Order of the particles by (cell key, id); ids None: the index is the id."""
    key = np.ascontiguousarray(key, dtype=np.int32)
    perm = np.zeros(len(key), dtype=np.int64)
    count = np.zeros(ncells, dtype=np.int64)
    start = np.zeros(ncells, dtype=np.int64)
    idp = None
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        idp = _ptr(ids, C.c_uint32)
    lib().orc_counting_sort(len(key), _ptr(key, C.c_int32), idp, ncells, _ptr(perm, C.c_int64),
                            _ptr(count, C.c_int64), _ptr(start, C.c_int64))
    return perm, count, start


def gather(perm, a):
    """out[j] = a[perm[j]] (rows of a contiguous array), by orc_gather."""
    a = np.ascontiguousarray(a)
    out = np.empty_like(a)
    width = a.itemsize * (a.size // len(a) if len(a) else 1)
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    lib().orc_gather(len(perm), _ptr(perm, C.c_int64), a.ctypes.data, out.ctypes.data, width)
    return out


def forces(cfg, x, flags, colloids):
    """Per-particle WCA force and total (fixed-point summed) colloid force."""
    p = make_params(cfg)
    x = np.ascontiguousarray(x, dtype=np.float64)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    nc = len(colloids["mass"])
    X = np.ascontiguousarray(colloids["x"], dtype=np.float64)
    f = np.zeros_like(x)
    F = np.zeros((nc, 3))
    lib().orc_forces(C.byref(p), len(x), _ptr(x, C.c_double), _ptr(flags, C.c_uint8), nc,
                     _ptr(X, C.c_double), _ptr(np.ascontiguousarray(colloids["sigma"], np.float64), C.c_double),
                     _ptr(np.ascontiguousarray(colloids["eps_A"], np.float64), C.c_double),
                     _ptr(np.ascontiguousarray(colloids["eps_B"], np.float64), C.c_double),
                     _ptr(f, C.c_double), _ptr(F, C.c_double))
    return f, F


def cc_forces(cfg, X, bonds=()):
    """Colloid-colloid LJ forces (fixed-point summed, bonded pairs excluded)."""
    p = make_params(cfg)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    ba = np.ascontiguousarray([b[0] for b in bonds], dtype=np.int32)
    bb = np.ascontiguousarray([b[1] for b in bonds], dtype=np.int32)
    F = np.zeros_like(X)
    lib().orc_cc_forces(C.byref(p), len(X), _ptr(X, C.c_double), len(ba), _ptr(ba, C.c_int32),
                        _ptr(bb, C.c_int32), _ptr(F, C.c_double))
    return F


# --------------------------------------------------------------------------
# rigid composite colloid (bead body)
# --------------------------------------------------------------------------
class Body:
    """Rigid bead body: centre of mass x, v; quaternion q (w, x, y, z, body ->
    space); body-frame angular momentum l; beads b[nb, 3] in the principal
    frame relative to x, each with eps_A, eps_B and a catalytic flag; bead
    mass and the common WCA sigma."""

    def __init__(self, d: dict):
        self.x = np.array(d["x"], dtype=np.float64).reshape(3)
        self.v = np.array(d["v"], dtype=np.float64).reshape(3)
        self.q = np.array(d["q"], dtype=np.float64).reshape(4)
        self.l = np.array(d["l"], dtype=np.float64).reshape(3)
        self.b = np.ascontiguousarray(d["b"], dtype=np.float64).reshape(-1, 3).copy()
        nb = len(self.b)
        self.epsA = np.ascontiguousarray(np.broadcast_to(d["eps_A"], nb), dtype=np.float64)
        self.epsB = np.ascontiguousarray(np.broadcast_to(d["eps_B"], nb), dtype=np.float64)
        self.cat = np.ascontiguousarray(np.broadcast_to(d["catalytic"], nb), dtype=np.int32)
        self.bead_mass = float(d["bead_mass"])
        self.sigma = float(d["sigma"])

    @property
    def nb(self) -> int:
        return len(self.b)

    def inertia(self):
        """(M, I[3]) from the beads."""
        M = C.c_double(0.0)
        I = np.zeros(3)
        lib().orc_body_inertia(self.nb, _ptr(self.b, C.c_double), self.bead_mass, C.byref(M), _ptr(I, C.c_double))
        return float(M.value), I

    def matrix(self) -> np.ndarray:
        return quat_matrix(self.q)

    def state(self) -> dict:
        return {"x": self.x.copy(), "v": self.v.copy(), "q": self.q.copy(), "l": self.l.copy()}


def quat_matrix(q) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros((3, 3))
    lib().orc_quat_matrix(_ptr(q, C.c_double), _ptr(R, C.c_double))
    return R


def body_rotate(I, dt, q, l, steps: int = 1):
    """Free rotation of a rigid body over `steps` sub-steps of dt (returns new q, l)."""
    I = np.ascontiguousarray(I, dtype=np.float64)
    q = np.array(q, dtype=np.float64)
    l = np.array(l, dtype=np.float64)
    for _ in range(steps):
        lib().orc_body_rotate(_ptr(I, C.c_double), dt, _ptr(q, C.c_double), _ptr(l, C.c_double))
    return q, l


def body_reach(b, sigma) -> float:
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(lib().orc_body_reach(len(b), _ptr(b, C.c_double), sigma))


def body_forces(cfg, x, flags, body: "Body"):
    """Solvent forces, body force, space torque and WCA energy of a configuration."""
    p = make_params(cfg)
    x = np.ascontiguousarray(x, dtype=np.float64)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    f = np.zeros_like(x)
    F = np.zeros(3)
    T = np.zeros(3)
    d = C.c_double
    e = lib().orc_body_forces(C.byref(p), len(x), _ptr(x, d), _ptr(flags, C.c_uint8), body.nb,
                              _ptr(body.b, d), _ptr(body.epsA, d), _ptr(body.epsB, d), _ptr(body.cat, C.c_int32),
                              body.sigma, _ptr(body.x, d), _ptr(body.q, d), _ptr(f, d), _ptr(F, d), _ptr(T, d))
    return f, F, T, float(e)


class SkinError(RuntimeError):
    """A colloid moved further than the skin during one interval."""


class OracleSystem:
    """One replica: solvent state (x, v, flags, id) in storage order, colloids and bonds.

    ``flags``: bit 0 = species B, bit 1 = catalytic tag.  ``id`` is carried so
    that permutations can be compared; it never enters the arithmetic except as
    the counter of the catalytic draw.
    """

    def __init__(self, cfg: dict, x, v, flags=None, ids=None, colloids=None, bonds=None, step: int = 0,
                 body=None, cell_order: str = "linear"):
        """cell_order: the order of the cells in storage -- "linear" (cell key
        order, x fastest) or "hilbert" (the compact Hilbert order of the
        collision grid, §1.2 / §1.4): only the storage order changes, every
        cell keeps its key (its linear index) for its draws and geometry."""
        self.cfg = dict(cfg)
        self.p = make_params(cfg)
        n = len(x)
        self.x = np.ascontiguousarray(x, dtype=np.float64).reshape(n, 3).copy()
        self.v = np.ascontiguousarray(v, dtype=np.float64).reshape(n, 3).copy()
        self.flags = (np.zeros(n, np.uint8) if flags is None else np.asarray(flags, np.uint8).copy())
        self.id = (np.arange(n, dtype=np.uint32) if ids is None else np.asarray(ids, np.uint32).copy())
        colloids = colloids or {"x": np.zeros((0, 3)), "v": np.zeros((0, 3)), "mass": [], "sigma": [],
                                "eps_A": [], "eps_B": [], "catalytic": []}
        self.X = np.ascontiguousarray(colloids["x"], dtype=np.float64).reshape(-1, 3).copy()
        self.V = np.ascontiguousarray(colloids["v"], dtype=np.float64).reshape(-1, 3).copy()
        self.M = np.ascontiguousarray(colloids["mass"], dtype=np.float64)
        self.sig = np.ascontiguousarray(colloids["sigma"], dtype=np.float64)
        self.epsA = np.ascontiguousarray(colloids["eps_A"], dtype=np.float64)
        self.epsB = np.ascontiguousarray(colloids["eps_B"], dtype=np.float64)
        self.cat = np.ascontiguousarray(colloids["catalytic"], dtype=np.int32)
        bonds = bonds or []
        self.ba = np.ascontiguousarray([b[0] for b in bonds], dtype=np.int32)
        self.bb = np.ascontiguousarray([b[1] for b in bonds], dtype=np.int32)
        self.bd = np.ascontiguousarray([b[2] for b in bonds], dtype=np.float64)
        self.body = None if body is None else Body(body)
        if self.body is not None and len(self.M):
            raise ValueError("a replica holds either colloids or one rigid body")
        self.step_index = int(step)
        self.ncells = int(lib().orc_n_cells(C.byref(self.p)))
        if cell_order not in ("linear", "hilbert"):
            raise ValueError(f"cell_order {cell_order!r}")
        self.cell_order = cell_order
        self.rank = None
        if cell_order == "hilbert":
            L = self.cfg["L"]
            nz = int(L[2]) + (1 if self.cfg.get("walls") else 0)
            self.rank = hilbert_rank((int(L[0]), int(L[1]), nz))
            if len(self.rank) != self.ncells:
                raise ValueError("Hilbert rank table does not cover the cells")
        self.key = None
        self.count = None
        self.start = None
        self.perm = None
        self.near = np.zeros(n, np.uint8)

    @property
    def n(self):
        return len(self.x)

    # -- the steps of one interval ------------------------------------------
    def interval(self, all_substep: bool = False) -> None:
        """Interval motion: MD sub-steps near colloids, free flight elsewhere."""
        L = lib()
        d, u8, u32, i32 = C.c_double, C.c_uint8, C.c_uint32, C.c_int32
        if self.body is not None:
            B = self.body
            rc = L.orc_interval_body(C.byref(self.p), self.step_index, self.n, _ptr(self.x, d), _ptr(self.v, d),
                                     _ptr(self.flags, u8), _ptr(self.id, u32), B.nb, _ptr(B.b, d),
                                     _ptr(B.epsA, d), _ptr(B.epsB, d), _ptr(B.cat, i32), B.bead_mass, B.sigma,
                                     _ptr(B.x, d), _ptr(B.v, d), _ptr(B.q, d), _ptr(B.l, d),
                                     1 if all_substep else 0, _ptr(self.near, u8))
            if rc != 0:
                raise SkinError("body displacement exceeded the skin")
            return
        nc = len(self.M)
        rc = L.orc_interval(C.byref(self.p), self.step_index, self.n, _ptr(self.x, d), _ptr(self.v, d),
                            _ptr(self.flags, u8), _ptr(self.id, u32), nc, _ptr(self.X, d), _ptr(self.V, d),
                            _ptr(self.M, d), _ptr(self.sig, d), _ptr(self.epsA, d), _ptr(self.epsB, d),
                            _ptr(self.cat, i32), len(self.ba), _ptr(self.ba, i32), _ptr(self.bb, i32),
                            _ptr(self.bd, d), 1 if all_substep else 0, _ptr(self.near, u8))
        if rc != 0:
            raise SkinError("colloid displacement exceeded the skin")

    def shift_and_sort(self) -> None:
        """Random grid shift, cell keys and counting sort by (cell, id); reorders the state."""
        L = lib()
        s = grid_shift(self.p.seed, self.step_index)
        key = np.zeros(self.n, dtype=np.int32)
        L.orc_cell_keys(C.byref(self.p), self.n, _ptr(self.x, C.c_double), _ptr(s, C.c_double),
                        _ptr(key, C.c_int32))
        if self.rank is None:
            perm, count, start = counting_sort(key, self.ncells, self.id)
        else:
            # storage by (Hilbert rank, id); count and start stay indexed by key
            perm, count_r, start_r = counting_sort(self.rank[key].astype(np.int32), self.ncells, self.id)
            count, start = count_r[self.rank], start_r[self.rank]
        self.x = gather(perm, self.x)
        self.v = gather(perm, self.v)
        self.flags = gather(perm, self.flags)
        self.id = gather(perm, self.id)
        self.near = gather(perm, self.near)
        self.key = gather(perm, key)
        self.perm, self.count, self.start = perm, count, start
        self.shift = s

    def collide(self) -> None:
        lib().orc_collide(C.byref(self.p), self.step_index, self.ncells, _ptr(self.count, C.c_int64),
                          _ptr(self.start, C.c_int64), _ptr(self.v, C.c_double))

    def react(self) -> None:
        lib().orc_bulk_react(C.byref(self.p), self.step_index, self.ncells, _ptr(self.count, C.c_int64),
                             _ptr(self.start, C.c_int64), _ptr(self.flags, C.c_uint8))

    def reservoirs(self) -> None:
        """Species reservoirs of the chemotactic set-up (cfg["reservoirs"] =
        ((ya0, ya1), (yb0, yb1)), y columns of the collision grid), if any."""
        res = self.cfg.get("reservoirs")
        if not res:
            return
        (ya0, ya1), (yb0, yb1) = res
        lib().orc_species_reservoirs(C.byref(self.p), self.ncells, _ptr(self.count, C.c_int64),
                                     _ptr(self.start, C.c_int64), _ptr(self.flags, C.c_uint8),
                                     int(ya0), int(ya1), int(yb0), int(yb1))

    def step(self, k: int = 1, all_substep: bool = False) -> None:
        """k full collision intervals."""
        for _ in range(k):
            self.interval(all_substep)
            self.shift_and_sort()
            self.collide()
            self.react()
            self.reservoirs()
            self.step_index += 1

    # -- observables ---------------------------------------------------------
    def temperature(self) -> float:
        """Cell-frame temperature of §1.4 on the current sort (cells with N >= 2)."""
        used = C.c_int64(0)
        return float(lib().orc_temperature(self.ncells, _ptr(self.count, C.c_int64),
                                           _ptr(self.start, C.c_int64), _ptr(self.v, C.c_double),
                                           C.byref(used)))

    def potential_energy(self) -> float:
        d, i32 = C.c_double, C.c_int32
        if self.body is not None:
            return body_forces(self.cfg, self.x, self.flags, self.body)[3]
        return float(lib().orc_potential_energy(
            C.byref(self.p), self.n, _ptr(self.x, d), _ptr(self.flags, C.c_uint8), len(self.M),
            _ptr(self.X, d), _ptr(self.sig, d), _ptr(self.epsA, d), _ptr(self.epsB, d),
            len(self.ba), _ptr(self.ba, i32), _ptr(self.bb, i32)))

    def kinetic_energy(self) -> float:
        e = 0.5 * float((self.v ** 2).sum()) + 0.5 * float((self.M[:, None] * self.V ** 2).sum())
        if self.body is not None:
            M, I = self.body.inertia()
            e += 0.5 * M * float(self.body.v @ self.body.v) + 0.5 * float((self.body.l ** 2 / I).sum())
        return e

    def momentum(self) -> np.ndarray:
        p = self.v.sum(0) + (self.M[:, None] * self.V).sum(0)
        if self.body is not None:
            p = p + self.body.inertia()[0] * self.body.v
        return p

    def colloids(self) -> dict:
        return {"x": self.X.copy(), "v": self.V.copy()}


# -- slab profile ----------------------------------------------------------------
def slab_profile(L_axis: int, x_axis, v, flags, n_bins: int) -> dict:
    """Slab histogram of the solvent along one axis: the flow profile of the
    Poiseuille set-up, the slab temperatures of the thermal-gradient set-up and
    the species profile of the chemotactic set-up (§"Applications of RMPCDMD";
    the histogram routine of the ``common`` module).

    Definition: particle i falls in bin floor(x_i * n_bins / L), clamped to
    [0, n_bins).  Per bin: the count, the count of species B (flag bit 0), the
    sum of v_k with every term first rounded (ties to even) to a multiple of
    2^-32, and the sum of v_k^2 with every term rounded to a multiple of 2^-24.
    The rounded terms are summed as exact integers."""
    x = np.asarray(x_axis, np.float64)
    v = np.asarray(v, np.float64).reshape(-1, 3)
    fl = np.zeros(len(x), np.uint8) if flags is None else np.asarray(flags, np.uint8)
    b = np.floor(x * float(n_bins) / float(L_axis))
    b = np.clip(b, 0, n_bins - 1).astype(np.int64)
    n = np.bincount(b, minlength=n_bins).astype(np.int64)
    nB = np.bincount(b, weights=(fl & 1).astype(np.float64), minlength=n_bins).astype(np.int64)
    s1 = np.zeros((n_bins, 3), np.int64)
    s2 = np.zeros((n_bins, 3), np.int64)
    for k in range(3):
        np.add.at(s1[:, k], b, np.rint(v[:, k] * 2.0 ** 32).astype(np.int64))
        np.add.at(s2[:, k], b, np.rint(v[:, k] * v[:, k] * 2.0 ** 24).astype(np.int64))
    return {"n": n, "n_B": nB, "v_sum": s1.astype(np.float64) * 2.0 ** -32,
            "v2_sum": s2.astype(np.float64) * 2.0 ** -24}


def slab_fields(p: dict) -> dict:
    """Mean flow u_b = v_sum / n and slab temperature (unit mass, the slab's
    own mean flow removed, N - 1 in the denominator as in the cell estimator
    of §1.4): T_b = sum_k (v2_sum_k - v_sum_k^2 / n) / (3 (n - 1)).  Bins with
    fewer than 2 particles give NaN."""
    n = p["n"].astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        u = p["v_sum"] / n[:, None]
        T = (p["v2_sum"] - p["v_sum"] ** 2 / n[:, None]).sum(1) / (3.0 * (n - 1.0))
    T[n < 2] = np.nan
    return {"u": u, "T": T, "c_B": np.where(n > 0, p["n_B"] / np.maximum(n, 1), np.nan)}


# -- linked bead network (iterative RATTLE) ---------------------------------------
def _links(links):
    la = np.ascontiguousarray([a for a, _ in links], dtype=np.int32)
    lb = np.ascontiguousarray([b for _, b in links], dtype=np.int32)
    return la, lb


def rattle_pos_iter(links, d, m, xold, x, v, dt, tol=1e-13, max_sweeps=10000):
    """Iterative RATTLE position stage (§1.4, Andersen 1983) on copies of x, v.
    Returns (x, v, sweeps); sweeps = -1 when the sweeps ran out."""
    la, lb = _links(links)
    d = np.ascontiguousarray(d, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    xold = np.ascontiguousarray(xold, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    dd = C.c_double
    n = lib().orc_rattle_pos_iter(len(la), _ptr(la, C.c_int32), _ptr(lb, C.c_int32), _ptr(d, dd), _ptr(m, dd),
                                  _ptr(xold, dd), _ptr(x, dd), _ptr(v, dd), dt, tol, max_sweeps)
    return x, v, int(n)


def rattle_vel_iter(links, d, m, x, v, tol=1e-13, max_sweeps=10000):
    """Iterative RATTLE velocity stage on a copy of v.  Returns (v, sweeps)."""
    la, lb = _links(links)
    d = np.ascontiguousarray(d, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    dd = C.c_double
    n = lib().orc_rattle_vel_iter(len(la), _ptr(la, C.c_int32), _ptr(lb, C.c_int32), _ptr(d, dd), _ptr(m, dd),
                                  _ptr(x, dd), _ptr(v, dd), tol, max_sweeps)
    return v, int(n)


def network_steps(links, d, m, x, v, dt, steps, F=None, tol=1e-13, max_sweeps=10000):
    """`steps` velocity-Verlet steps of a linked bead network (forces F held
    fixed, or none).  Returns (x, v, largest sweep count or -1)."""
    la, lb = _links(links)
    d = np.ascontiguousarray(d, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    Fp = None if F is None else _ptr(np.ascontiguousarray(F, dtype=np.float64), C.c_double)
    dd = C.c_double
    worst = 0
    for _ in range(steps):
        n = lib().orc_network_step(len(m), _ptr(m, dd), len(la), _ptr(la, C.c_int32), _ptr(lb, C.c_int32),
                                   _ptr(d, dd), Fp, _ptr(x, dd), _ptr(v, dd), dt, tol, max_sweeps)
        if n < 0:
            return x, v, -1
        worst = max(worst, n)
    return x, v, worst


class Network:
    """Janus particle as beads held at fixed distances by iterative RATTLE:
    bead positions xb (unwrapped) and velocities vb, masses mb, eps_A, eps_B,
    catalytic flags, the common WCA sigma, links [(a, b)] of lengths d."""

    def __init__(self, xb, vb, mb, epsA, epsB, cat, sigma, links, d):
        self.xb = np.array(xb, dtype=np.float64).reshape(-1, 3)
        self.vb = np.array(vb, dtype=np.float64).reshape(-1, 3)
        nb = len(self.xb)
        self.mb = np.ascontiguousarray(np.broadcast_to(mb, nb), dtype=np.float64)
        self.epsA = np.ascontiguousarray(np.broadcast_to(epsA, nb), dtype=np.float64)
        self.epsB = np.ascontiguousarray(np.broadcast_to(epsB, nb), dtype=np.float64)
        self.cat = np.ascontiguousarray(np.broadcast_to(cat, nb), dtype=np.int32)
        self.sigma = float(sigma)
        self.la, self.lb = _links(links)
        self.d = np.ascontiguousarray(d, dtype=np.float64)

    @classmethod
    def from_body(cls, body, links, d):
        """The beads of a rigid-body description (dict or Body) moving with it."""
        B = body if isinstance(body, Body) else Body(body)
        R = quat_matrix(B.q)
        _, I = B.inertia()
        r = B.b @ R.T
        w = R @ (B.l / I)
        return cls(B.x + r, B.v + np.cross(w, r), B.bead_mass, B.epsA, B.epsB, B.cat, B.sigma, links, d)

    def momentum(self) -> np.ndarray:
        return (self.mb[:, None] * self.vb).sum(0)

    def kinetic_energy(self) -> float:
        return 0.5 * float((self.mb[:, None] * self.vb ** 2).sum())

    def com(self) -> np.ndarray:
        return (self.mb[:, None] * self.xb).sum(0) / self.mb.sum()


def interval_network(cfg, x, v, flags, ids, net: Network, step: int = 0, all_substep: bool = False,
                     tol: float = 1e-12, max_sweeps: int = 10000):
    """One interval of solvent + bead network (in place).  Returns (status,
    near mask): status 0, 1 (centre of mass beyond the skin) or 2 (RATTLE did
    not converge)."""
    p = make_params(cfg)
    dd, u8, u32, i32 = C.c_double, C.c_uint8, C.c_uint32, C.c_int32
    n = len(x)
    near = np.zeros(max(n, 1), dtype=np.uint8)
    rc = lib().orc_interval_network(C.byref(p), step, n, _ptr(x, dd), _ptr(v, dd), _ptr(flags, u8), _ptr(ids, u32),
                                    len(net.mb), _ptr(net.xb, dd), _ptr(net.vb, dd), _ptr(net.mb, dd),
                                    _ptr(net.epsA, dd), _ptr(net.epsB, dd), _ptr(net.cat, i32), net.sigma,
                                    len(net.la), _ptr(net.la, i32), _ptr(net.lb, i32), _ptr(net.d, dd), tol,
                                    max_sweeps, 1 if all_substep else 0, _ptr(near, u8))
    return int(rc), near[:n].astype(bool)


def network_energy(cfg, x, flags, net: Network) -> float:
    """WCA energy between the solvent and the beads."""
    p = make_params(cfg)
    dd = C.c_double
    x = np.ascontiguousarray(x, dtype=np.float64)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    return float(lib().orc_network_energy(C.byref(p), len(x), _ptr(x, dd), _ptr(flags, C.c_uint8), len(net.mb),
                                          _ptr(net.xb, dd), _ptr(net.epsA, dd), _ptr(net.epsB, dd),
                                          _ptr(net.cat, C.c_int32), net.sigma))


# -- Hilbert order of the cells ----------------------------------------------------
def hilbert_index(m: int, x: int, y: int, z: int) -> int:
    """Index of cell (x, y, z) on the 3-D Hilbert curve through the 2^m cube."""
    return int(lib().orc_hilbert_index(int(m), int(x), int(y), int(z)))


def hilbert_rank(L) -> np.ndarray:
    """Place of every cell c = x + L0 (y + L1 z) in the Hilbert order of the box."""
    Lc = np.ascontiguousarray([int(a) for a in L], dtype=np.int32)
    rank = np.zeros(int(np.prod(Lc)), dtype=np.int64)
    if lib().orc_hilbert_rank(_ptr(Lc, C.c_int32), _ptr(rank, C.c_int64)) != 0:
        raise MemoryError("hilbert_rank")
    return rank
