"""Thin ctypes binding of the C ABI in ``include/rmpcd.h`` (argument marshalling only).

Every step of the collision interval runs in the CUDA kernels of
``_build/librmpcd.so``; if that library is missing this module raises -- there
is no CPU path.  PyTorch is used only for device buffers and the current CUDA
stream when it is available.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RMPCD_FP64 = 0
RMPCD_MIXED = 1

STATUS = {0: "OK", 1: "EINVAL", 2: "ECUDA", 3: "ENOMEM", 4: "EOVERFLOW", 5: "ESKIN", 6: "ETIMEOUT", 7: "ESTATE"}


def cell_places(dims, order="hilbert"):
    """rmpcd_cell_places: the place of every cell key of a grid (host call)."""
    L = load()
    d = (C.c_int32 * 3)(*[int(a) for a in dims])
    n = int(dims[0]) * int(dims[1]) * int(dims[2])
    out = np.zeros(n, dtype=np.int64)
    st = L.rmpcd_cell_places(d, CELL_ORDERS[order], out.ctypes.data_as(C.POINTER(C.c_int64)))
    if st != 0:
        raise RmpcdError(st, "rmpcd_cell_places")
    return out


class RmpcdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"rmpcd {STATUS.get(status, status)}: {message}")
        self.status = status
        self.code = STATUS.get(status, str(status))


class Params(C.Structure):
    _fields_ = [
        ("L", C.c_int32 * 3), ("walls", C.c_int32), ("rho_wall", C.c_int32), ("n_md", C.c_int32),
        ("n_slabs", C.c_int32), ("n_solvent", C.c_int32), ("n_colloids", C.c_int32), ("n_bonds", C.c_int32),
        ("kT", C.c_double), ("alpha", C.c_double), ("tau", C.c_double), ("g", C.c_double * 3),
        ("bulk_rate", C.c_double), ("cat_prob", C.c_double), ("skin", C.c_double),
        ("slab_x0", C.c_double * 4), ("slab_x1", C.c_double * 4), ("slab_kT", C.c_double * 4),
        ("cc_eps", C.c_double), ("cc_sigma", C.c_double), ("cc_rc", C.c_double), ("seed", C.c_uint64),
        ("res_y", C.c_int32 * 4),
    ]


class Colloid(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("v", C.c_double * 3), ("mass", C.c_double), ("sigma", C.c_double),
                ("eps_A", C.c_double), ("eps_B", C.c_double), ("catalytic", C.c_int32), ("pad", C.c_int32)]


class Bond(C.Structure):
    _fields_ = [("a", C.c_int32), ("b", C.c_int32), ("d", C.c_double)]


class Body(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("v", C.c_double * 3), ("q", C.c_double * 4), ("l", C.c_double * 3),
                ("bead_mass", C.c_double), ("sigma", C.c_double), ("n_beads", C.c_int32), ("pad", C.c_int32)]


class Bead(C.Structure):
    _fields_ = [("b", C.c_double * 3), ("eps_A", C.c_double), ("eps_B", C.c_double), ("catalytic", C.c_int32),
                ("pad", C.c_int32)]


MAX_BEADS = 1024


class NetBead(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("v", C.c_double * 3), ("mass", C.c_double), ("eps_A", C.c_double),
                ("eps_B", C.c_double), ("catalytic", C.c_int32), ("pad", C.c_int32)]


MAX_NET_BEADS = 512


class Obs(C.Structure):
    _fields_ = [("temperature", C.c_double), ("momentum", C.c_double * 3), ("kinetic", C.c_double),
                ("n_cells_used", C.c_int64), ("n_B", C.c_int64), ("n_solvent", C.c_int64),
                ("step", C.c_uint32), ("pad", C.c_uint32)]


MAX_PROFILE_BINS = 512


class ProfileBin(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_B", C.c_int64), ("v_sum", C.c_double * 3), ("v2_sum", C.c_double * 3)]


class Timers(C.Structure):
    _fields_ = [("launches", C.c_int64 * 4), ("ms", C.c_double * 4)]


PHASES = ("prime", "md", "cellpass", "obs")

EXPORTS = [
    "rmpcd_create", "rmpcd_destroy", "rmpcd_set_state", "rmpcd_get_state", "rmpcd_set_colloids",
    "rmpcd_get_colloids", "rmpcd_set_step", "rmpcd_get_step", "rmpcd_stream", "rmpcd_shift_and_sort",
    "rmpcd_collide", "rmpcd_react", "rmpcd_step", "rmpcd_observables", "rmpcd_sync", "rmpcd_launch_count",
    "rmpcd_last_error", "rmpcd_enable_timers", "rmpcd_read_timers", "rmpcd_set_tuning", "rmpcd_get_tuning",
    "rmpcd_observables_noalloc", "rmpcd_set_graphs", "rmpcd_get_bucket_cap", "rmpcd_set_body", "rmpcd_get_body",
    "rmpcd_profile", "rmpcd_workspace_size", "rmpcd_set_wait_test", "rmpcd_md_substep", "rmpcd_set_network",
    "rmpcd_get_network", "rmpcd_set_state_all", "rmpcd_get_state_all", "rmpcd_set_cell_order",
    "rmpcd_get_cell_order", "rmpcd_cell_places",
]
CELL_ORDERS = {"linear": 0, "hilbert": 1}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load librmpcd.so (built by ``build.build()``); raise if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (paper_1608_04904_gb300.build.build())")
    L = C.CDLL(path)
    P = C.POINTER
    vp, i32, i64, u32, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
    L.rmpcd_create.argtypes = [P(vp), i32, i32, P(Params), P(Colloid), P(Bond), i32, vp]
    L.rmpcd_set_wait_test.argtypes = [vp, i32, i32]
    L.rmpcd_md_substep.argtypes = [vp, i32]
    L.rmpcd_set_network.argtypes = [vp, i32, P(NetBead), i32, P(Bond), P(i32), i32, d, d, i32]
    L.rmpcd_get_network.argtypes = [vp, i32, P(d), P(d), i32]
    L.rmpcd_destroy.argtypes = [vp]
    L.rmpcd_destroy.restype = None
    L.rmpcd_set_state.argtypes = [vp, i32, vp, vp, vp, i64, i32]
    L.rmpcd_get_state.argtypes = [vp, i32, vp, vp, vp, vp, vp, i64, i32]
    L.rmpcd_set_state_all.argtypes = [vp, vp, vp, vp, i64, i32]
    L.rmpcd_set_cell_order.argtypes = [vp, i32]
    L.rmpcd_get_cell_order.argtypes = [vp, P(i32)]
    L.rmpcd_cell_places.argtypes = [P(i32), i32, P(i64)]
    L.rmpcd_get_state_all.argtypes = [vp, vp, vp, vp, vp, vp, i64, i32]
    L.rmpcd_set_colloids.argtypes = [vp, i32, P(Colloid), i32]
    L.rmpcd_get_colloids.argtypes = [vp, i32, P(Colloid), i32]
    L.rmpcd_set_body.argtypes = [vp, i32, P(Body), P(Bead)]
    L.rmpcd_get_body.argtypes = [vp, i32, P(Body)]
    L.rmpcd_set_step.argtypes = [vp, u32]
    L.rmpcd_get_step.argtypes = [vp, P(u32)]
    for name in ("rmpcd_stream", "rmpcd_shift_and_sort", "rmpcd_collide", "rmpcd_react", "rmpcd_sync"):
        getattr(L, name).argtypes = [vp]
    L.rmpcd_step.argtypes = [vp, i32]
    L.rmpcd_observables.argtypes = [vp, i32, P(Obs)]
    L.rmpcd_profile.argtypes = [vp, i32, i32, i32, P(ProfileBin)]
    L.rmpcd_workspace_size.argtypes = [i32, i32, P(Params), P(Colloid), P(Bond), i32, P(C.c_size_t)]
    L.rmpcd_launch_count.argtypes = [vp, P(i64)]
    L.rmpcd_enable_timers.argtypes = [vp, i32]
    L.rmpcd_read_timers.argtypes = [vp, P(Timers), i32]
    L.rmpcd_set_tuning.argtypes = [vp, i32, i32]
    L.rmpcd_set_graphs.argtypes = [vp, i32]
    L.rmpcd_get_bucket_cap.argtypes = [vp, P(i32)]
    L.rmpcd_get_tuning.argtypes = [vp, P(i32), P(i32)]
    L.rmpcd_observables_noalloc.argtypes = [vp, vp, vp, i64, i32, vp, vp]
    L.rmpcd_last_error.argtypes = [vp]
    L.rmpcd_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("rmpcd_destroy", "rmpcd_last_error"):
            getattr(L, name).restype = C.c_int
    _LIB = L
    return L


def make_params(cfg: dict, n_solvent: int, n_colloids: int = 0, n_bonds: int = 0) -> Params:
    p = Params()
    p.L[:] = [int(a) for a in cfg["L"]]
    p.walls = int(cfg.get("walls", 0))
    p.rho_wall = int(cfg.get("rho_wall", 0))
    p.n_md = int(cfg.get("n_md", 1))
    slabs = cfg.get("slabs", []) or []
    p.n_slabs = len(slabs)
    for k, (x0, x1, kt) in enumerate(slabs):
        p.slab_x0[k], p.slab_x1[k], p.slab_kT[k] = x0, x1, kt
    p.n_solvent = int(n_solvent)
    p.n_colloids = int(n_colloids)
    p.n_bonds = int(n_bonds)
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
    res = cfg.get("reservoirs")
    if res:
        (ya0, ya1), (yb0, yb1) = res
        p.res_y[:] = [int(ya0), int(ya1), int(yb0), int(yb1)]
    return p


def _colloid(c) -> Colloid:
    o = Colloid()
    o.x[:] = [float(a) for a in c["x"]]
    o.v[:] = [float(a) for a in c.get("v", (0.0, 0.0, 0.0))]
    o.mass, o.sigma = float(c["mass"]), float(c["sigma"])
    o.eps_A, o.eps_B = float(c["eps_A"]), float(c["eps_B"])
    o.catalytic = int(c.get("catalytic", 0))
    return o


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


def _marshal(replicas):
    """Params, colloid and bond arrays of rmpcd_create for a list of replicas."""
    n = len(replicas)
    params = (Params * n)()
    cols, bonds = [], []
    for r, rep in enumerate(replicas):
        cl = list(rep.get("colloids", []) or [])
        bl = list(rep.get("bonds", []) or [])
        params[r] = make_params(rep["cfg"], rep["n"], len(cl), len(bl))
        cols += [_colloid(c) for c in cl]
        for a, b, dd in bl:
            bo = Bond()
            bo.a, bo.b, bo.d = int(a), int(b), float(dd)
            bonds.append(bo)
    carr = (Colloid * max(1, len(cols)))(*cols)
    barr = (Bond * max(1, len(bonds)))(*bonds)
    return params, carr, barr, cols, bonds


def workspace_size(replicas, precision: str = "mixed", bucket_cap: int = 64) -> int:
    """rmpcd_workspace_size: device bytes System(replicas, precision, bucket_cap)
    would allocate (no GPU needed)."""
    L = load()
    params, carr, barr, cols, bonds = _marshal(list(replicas))
    out = C.c_size_t(0)
    prec = RMPCD_MIXED if precision == "mixed" else RMPCD_FP64
    st = L.rmpcd_workspace_size(prec, len(replicas), params, carr if cols else None, barr if bonds else None,
                                int(bucket_cap), C.byref(out))
    if st != 0:
        raise RmpcdError(st, L.rmpcd_last_error(None).decode())
    return int(out.value)


class System:
    """A set of independent replicas on the current CUDA device.

    ``replicas``: list of dicts with keys ``cfg`` (parameter dict), ``n``
    (solvent count), ``colloids`` (list of dicts), ``bonds`` (list of
    ``(a, b, d)``) and optionally ``body`` (a rigid bead body, see
    ``set_body``; such a replica has no colloids).
    """

    def __init__(self, replicas, precision: str = "mixed", bucket_cap: int = 64, stream=None):
        self._lib = load()
        self.precision = precision
        self.replicas = list(replicas)
        n = len(self.replicas)
        params, carr, barr, cols, bonds = _marshal(self.replicas)
        self.n = [int(rep["n"]) for rep in self.replicas]
        self.n_col = [len(list(rep.get("colloids", []) or [])) for rep in self.replicas]
        if stream is None:
            stream = _default_stream()
        elif hasattr(stream, "cuda_stream"):
            stream = int(stream.cuda_stream)
        self.stream = int(stream)
        handle = C.c_void_p()
        prec = RMPCD_MIXED if precision == "mixed" else RMPCD_FP64
        st = self._lib.rmpcd_create(C.byref(handle), prec, n, params, carr if cols else None,
                                    barr if bonds else None, int(bucket_cap), C.c_void_p(self.stream))
        if st != 0:
            raise RmpcdError(st, self._lib.rmpcd_last_error(None).decode())
        self._h = handle
        for r, rep in enumerate(self.replicas):
            if rep.get("body") is not None:
                self.set_body(r, rep["body"])

    @classmethod
    def single(cls, cfg, n, colloids=(), bonds=(), precision=None, bucket_cap=None, stream=None):
        precision = precision or cfg.get("precision", "mixed")
        bucket_cap = cfg.get("bucket_cap", 64) if bucket_cap is None else bucket_cap
        return cls([dict(cfg=cfg, n=n, colloids=list(colloids), bonds=list(bonds))], precision, bucket_cap, stream)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.rmpcd_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st != 0:
            raise RmpcdError(st, self._lib.rmpcd_last_error(self._h).decode())

    # -- state ---------------------------------------------------------------
    def set_state(self, replica, x, v, flags=None):
        n = self.n[replica]
        if _is_torch(x) and x.is_cuda:
            import torch
            x = x.contiguous().to(torch.float64)
            v = v.contiguous().to(torch.float64)
            f = None if flags is None else flags.contiguous().to(torch.uint8)
            self._keep = (x, v, f)
            self._check(self._lib.rmpcd_set_state(self._h, replica, C.c_void_p(x.data_ptr()),
                                                  C.c_void_p(v.data_ptr()),
                                                  None if f is None else C.c_void_p(f.data_ptr()), n, 1))
            return
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(n, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(n, 3)
        f = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8).reshape(n)
        self._check(self._lib.rmpcd_set_state(self._h, replica, x.ctypes.data_as(C.c_void_p),
                                              v.ctypes.data_as(C.c_void_p),
                                              None if f is None else f.ctypes.data_as(C.c_void_p), n, 0))

    def get_state(self, replica=0, out=None):
        """Return dict x, v, flags, id, cell (numpy arrays); with ``out`` (a dict
        of preallocated arrays, host numpy or CUDA torch tensors) fill those."""
        n = self.n[replica]
        if out is not None and any(_is_torch(a) and a.is_cuda for a in out.values()):
            ptr = lambda k: C.c_void_p(out[k].data_ptr()) if k in out else None
            self._check(self._lib.rmpcd_get_state(self._h, replica, ptr("x"), ptr("v"), ptr("flags"), ptr("id"),
                                                  ptr("cell"), n, 1))
            return out
        if out is None:
            out = {"x": np.empty((n, 3)), "v": np.empty((n, 3)), "flags": np.empty(n, np.uint8),
                   "id": np.empty(n, np.uint32), "cell": np.empty(n, np.int32)}
        ptr = lambda k: out[k].ctypes.data_as(C.c_void_p) if k in out else None
        self._check(self._lib.rmpcd_get_state(self._h, replica, ptr("x"), ptr("v"), ptr("flags"), ptr("id"),
                                              ptr("cell"), n, 0))
        return out

    def set_state_all(self, x, v, flags=None):
        """rmpcd_set_state_all: every replica's solvent in one call, the arrays
        concatenated in replica order (numpy host arrays or CUDA tensors)."""
        n = int(sum(self.n))
        if _is_torch(x) and x.is_cuda:
            import torch
            x = x.contiguous().to(torch.float64)
            v = v.contiguous().to(torch.float64)
            f = None if flags is None else flags.contiguous().to(torch.uint8)
            self._keep = (x, v, f)
            self._check(self._lib.rmpcd_set_state_all(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(v.data_ptr()),
                                                      None if f is None else C.c_void_p(f.data_ptr()), n, 1))
            return
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(n, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(n, 3)
        f = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8).reshape(n)
        self._check(self._lib.rmpcd_set_state_all(self._h, x.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p),
                                                  None if f is None else f.ctypes.data_as(C.c_void_p), n, 0))

    def get_state_all(self, out=None):
        """rmpcd_get_state_all: every replica's solvent, concatenated in replica
        order; ``out`` as for get_state (host numpy or CUDA torch arrays)."""
        n = int(sum(self.n))
        if out is not None and any(_is_torch(a) and a.is_cuda for a in out.values()):
            ptr = lambda k: C.c_void_p(out[k].data_ptr()) if k in out else None
            self._check(self._lib.rmpcd_get_state_all(self._h, ptr("x"), ptr("v"), ptr("flags"), ptr("id"),
                                                      ptr("cell"), n, 1))
            return out
        if out is None:
            out = {"x": np.empty((n, 3)), "v": np.empty((n, 3)), "flags": np.empty(n, np.uint8),
                   "id": np.empty(n, np.uint32), "cell": np.empty(n, np.int32)}
        ptr = lambda k: out[k].ctypes.data_as(C.c_void_p) if k in out else None
        self._check(self._lib.rmpcd_get_state_all(self._h, ptr("x"), ptr("v"), ptr("flags"), ptr("id"),
                                                  ptr("cell"), n, 0))
        return out

    def set_cell_order(self, order):
        """rmpcd_set_cell_order: "linear" (cell key order) or "hilbert"."""
        self._check(self._lib.rmpcd_set_cell_order(self._h, CELL_ORDERS[order]))

    def get_cell_order(self):
        o = C.c_int32(-1)
        self._check(self._lib.rmpcd_get_cell_order(self._h, C.byref(o)))
        return {v: k for k, v in CELL_ORDERS.items()}[o.value]

    def set_colloids(self, replica, colloids):
        arr = (Colloid * max(1, len(colloids)))(*[_colloid(c) for c in colloids])
        self._check(self._lib.rmpcd_set_colloids(self._h, replica, arr, len(colloids)))

    def get_colloids(self, replica=0):
        k = self.n_col[replica]
        arr = (Colloid * max(1, k))()
        self._check(self._lib.rmpcd_get_colloids(self._h, replica, arr, k))
        return {"x": np.array([list(arr[j].x) for j in range(k)]).reshape(k, 3),
                "v": np.array([list(arr[j].v) for j in range(k)]).reshape(k, 3)}

    def set_body(self, replica, body):
        """Rigid bead body of one replica: dict with x, v (centre of mass), q
        (w, x, y, z), l (body-frame angular momentum), b[nb, 3] (principal
        frame), eps_A, eps_B (per bead or scalar), catalytic (per bead or
        scalar), bead_mass, sigma."""
        b = np.ascontiguousarray(body["b"], dtype=np.float64).reshape(-1, 3)
        nb = len(b)
        eA = np.broadcast_to(np.asarray(body["eps_A"], np.float64), nb)
        eB = np.broadcast_to(np.asarray(body["eps_B"], np.float64), nb)
        cat = np.broadcast_to(np.asarray(body["catalytic"], np.int32), nb)
        B = Body()
        B.x[:] = [float(a) for a in body["x"]]
        B.v[:] = [float(a) for a in body["v"]]
        B.q[:] = [float(a) for a in body["q"]]
        B.l[:] = [float(a) for a in body["l"]]
        B.bead_mass = float(body["bead_mass"])
        B.sigma = float(body["sigma"])
        B.n_beads = nb
        beads = (Bead * max(1, nb))()
        for j in range(nb):
            beads[j].b[:] = [float(a) for a in b[j]]
            beads[j].eps_A = float(eA[j])
            beads[j].eps_B = float(eB[j])
            beads[j].catalytic = int(cat[j])
        self._check(self._lib.rmpcd_set_body(self._h, replica, C.byref(B), beads))

    def set_network(self, replica, xb, vb, mb, eps_A, eps_B, catalytic, sigma, links, d, colors, tol=1e-12,
                    max_sweeps=10000):
        """rmpcd_set_network: a bead network held by iterative RATTLE (FP64
        systems).  xb, vb [nb, 3] (box frame, unwrapped); mb, eps_A, eps_B,
        catalytic per bead or scalar; links [(a, b)] of lengths d with an
        edge colouring `colors` (no bead twice in a colour)."""
        xb = np.ascontiguousarray(xb, dtype=np.float64).reshape(-1, 3)
        vb = np.ascontiguousarray(vb, dtype=np.float64).reshape(-1, 3)
        nb = len(xb)
        mb = np.broadcast_to(np.asarray(mb, np.float64), nb)
        eA = np.broadcast_to(np.asarray(eps_A, np.float64), nb)
        eB = np.broadcast_to(np.asarray(eps_B, np.float64), nb)
        cat = np.broadcast_to(np.asarray(catalytic, np.int32), nb)
        beads = (NetBead * max(1, nb))()
        for j in range(nb):
            beads[j].x[:] = [float(a) for a in xb[j]]
            beads[j].v[:] = [float(a) for a in vb[j]]
            beads[j].mass, beads[j].eps_A, beads[j].eps_B = float(mb[j]), float(eA[j]), float(eB[j])
            beads[j].catalytic = int(cat[j])
        nl = len(links)
        la = (Bond * max(1, nl))()
        for k, (a, b) in enumerate(links):
            la[k].a, la[k].b, la[k].d = int(a), int(b), float(d[k])
        col = (C.c_int32 * max(1, nl))(*[int(c) for c in colors])
        self._check(self._lib.rmpcd_set_network(self._h, int(replica), beads, nb, la, col, nl, float(sigma),
                                                float(tol), int(max_sweeps)))
        self._net_nb = getattr(self, "_net_nb", {})
        self._net_nb[int(replica)] = nb

    def get_network(self, replica=0):
        """Bead positions and velocities of a replica's network: (x, v)."""
        nb = self._net_nb[int(replica)]
        x = np.empty((nb, 3))
        v = np.empty((nb, 3))
        self._check(self._lib.rmpcd_get_network(self._h, int(replica), x.ctypes.data_as(C.POINTER(C.c_double)),
                                                v.ctypes.data_as(C.POINTER(C.c_double)), nb))
        return x, v

    def get_body(self, replica=0) -> dict:
        """State of a replica's body: x, v, q, l (numpy arrays)."""
        B = Body()
        self._check(self._lib.rmpcd_get_body(self._h, replica, C.byref(B)))
        return {"x": np.array(list(B.x)), "v": np.array(list(B.v)), "q": np.array(list(B.q)),
                "l": np.array(list(B.l))}

    def set_step(self, step):
        self._check(self._lib.rmpcd_set_step(self._h, int(step)))

    def get_step(self):
        s = C.c_uint32()
        self._check(self._lib.rmpcd_get_step(self._h, C.byref(s)))
        return int(s.value)

    # -- the steps -----------------------------------------------------------
    def stream_interval(self):
        self._check(self._lib.rmpcd_stream(self._h))

    def md_substep(self, k):
        """rmpcd_md_substep: sub-step k of the current interval (in order from 0)."""
        self._check(self._lib.rmpcd_md_substep(self._h, int(k)))

    def shift_and_sort(self):
        self._check(self._lib.rmpcd_shift_and_sort(self._h))

    def collide(self):
        self._check(self._lib.rmpcd_collide(self._h))

    def react(self):
        self._check(self._lib.rmpcd_react(self._h))

    def step(self, n=1):
        self._check(self._lib.rmpcd_step(self._h, int(n)))

    def sync(self):
        self._check(self._lib.rmpcd_sync(self._h))

    def observables(self, replica=0) -> dict:
        o = Obs()
        self._check(self._lib.rmpcd_observables(self._h, replica, C.byref(o)))
        return {"temperature": o.temperature, "momentum": np.array(list(o.momentum)), "kinetic": o.kinetic,
                "n_cells_used": int(o.n_cells_used), "n_B": int(o.n_B), "n_solvent": int(o.n_solvent),
                "step": int(o.step)}

    def profile(self, replica=0, axis=2, n_bins=None) -> dict:
        """rmpcd_profile: per-bin solvent count, B count and fixed-point sums of
        v_k and v_k^2 along `axis` (n_bins defaults to one bin per cell)."""
        if n_bins is None:
            n_bins = int(self.replicas[replica]["cfg"]["L"][axis])
        out = (ProfileBin * max(int(n_bins), 1))()
        self._check(self._lib.rmpcd_profile(self._h, replica, int(axis), int(n_bins), out))
        a = np.frombuffer(out, dtype=np.dtype([("n", "<i8"), ("n_B", "<i8"), ("v_sum", "<f8", 3),
                                                ("v2_sum", "<f8", 3)]))
        return {"n": a["n"].copy(), "n_B": a["n_B"].copy(), "v_sum": a["v_sum"].copy(),
                "v2_sum": a["v2_sum"].copy()}

    def enable_timers(self, on=True):
        self._check(self._lib.rmpcd_enable_timers(self._h, 1 if on else 0))

    def read_timers(self, reset=True) -> dict:
        t = Timers()
        self._check(self._lib.rmpcd_read_timers(self._h, C.byref(t), 1 if reset else 0))
        return {name: {"launches": int(t.launches[k]), "ms": float(t.ms[k])} for k, name in enumerate(PHASES)}

    def set_tuning(self, md_cluster=0, md_kernel=0):
        self._check(self._lib.rmpcd_set_tuning(self._h, int(md_cluster), int(md_kernel)))

    def bucket_cap(self) -> int:
        c = C.c_int32()
        self._check(self._lib.rmpcd_get_bucket_cap(self._h, C.byref(c)))
        return int(c.value)

    def set_wait_test(self, max_polls=0, stall=False):
        """rmpcd_set_wait_test: the look-back wait's poll limit (0 = default)
        and the stall hook that makes every wait run out (tests only)."""
        self._check(self._lib.rmpcd_set_wait_test(self._h, int(max_polls), 1 if stall else 0))

    def set_graphs(self, on=True):
        self._check(self._lib.rmpcd_set_graphs(self._h, 1 if on else 0))

    def get_tuning(self):
        """(md_cluster, md_kernel) in use; md_cluster is 0 while tuning."""
        c, k = C.c_int32(), C.c_int32()
        self._check(self._lib.rmpcd_get_tuning(self._h, C.byref(c), C.byref(k)))
        return int(c.value), int(k.value)

    def launch_count(self) -> int:
        c = C.c_int64()
        self._check(self._lib.rmpcd_launch_count(self._h, C.byref(c)))
        return int(c.value)


RMPCD_NOALLOC_MAX_CELLS = 65536


def _check_noalloc_args(cell, v, flags, out) -> None:
    """The C entry point sees raw pointers only: check dtypes, shapes, layout
    and device here, so that no kernel reads or writes past a tensor."""
    import torch
    named = [("cell", cell, torch.int32), ("v", v, torch.float64), ("out", out, torch.float64)]
    if flags is not None:
        named.append(("flags", flags, torch.uint8))
    for name, t, dt in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch.Tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    n = int(cell.numel())
    if cell.dim() != 1:
        raise ValueError(f"cell must be 1-D, got shape {tuple(cell.shape)}")
    if tuple(v.shape) != (n, 3):
        raise ValueError(f"v must have shape ({n}, 3), got {tuple(v.shape)}")
    if flags is not None and int(flags.numel()) != n:
        raise ValueError(f"flags must have {n} entries, got {int(flags.numel())}")
    if int(out.numel()) < 8:
        raise ValueError(f"out must hold at least 8 doubles, got {int(out.numel())}")
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    for name, t, _ in named:
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")


def observables_noalloc(cell, v, flags, n_cells: int, out, stream=None) -> None:
    """rmpcd_observables_noalloc on CUDA tensors: cell (int32, n), v (float64,
    n x 3), flags (uint8, n, or None) and out (float64, 8), all contiguous on
    the current device.  Queued on ``stream`` (default: torch's current
    stream); out = [T, px, py, pz, kinetic, N_c, N_B, n counted]."""
    _check_noalloc_args(cell, v, flags, out)
    L = load()
    n = int(cell.numel())
    st = L.rmpcd_observables_noalloc(C.c_void_p(cell.data_ptr()), C.c_void_p(v.data_ptr()),
                                     None if flags is None else C.c_void_p(flags.data_ptr()), n, int(n_cells),
                                     C.c_void_p(out.data_ptr()),
                                     C.c_void_p(_default_stream() if stream is None else int(stream)))
    if st != 0:
        raise RmpcdError(st, L.rmpcd_last_error(None).decode())
