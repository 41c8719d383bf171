"""rmpcd_observables_noalloc: the observables reduction through static device
scratch (no device allocation), compared with rmpcd_observables on the same
state.  The file name sorts last so that the GPU case also runs after every
other test has used the device."""
import ctypes as C

import numpy as np
import pytest

from paper_1608_04904_gb300 import api, build, synth


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.load()


def test_rejects_sizes_beyond_the_static_limit(lib):
    """Host-side checks run before any CUDA call, so this runs without a GPU."""
    out = C.c_void_p(8)
    for n_cells in (0, api.RMPCD_NOALLOC_MAX_CELLS + 1):
        st = lib.rmpcd_observables_noalloc(None, None, None, 0, n_cells, out, None)
        assert api.STATUS[st] == "EINVAL"
        msg = lib.rmpcd_last_error(None).decode()
        assert "n_cells" in msg and str(api.RMPCD_NOALLOC_MAX_CELLS) in msg, msg
    st = lib.rmpcd_observables_noalloc(None, None, None, -1, 16, out, None)
    assert api.STATUS[st] == "EINVAL"
    st = lib.rmpcd_observables_noalloc(None, None, None, 0, 16, None, None)
    assert api.STATUS[st] == "EINVAL"


def _system(kind, precision):
    if kind == "sphere16":
        cfg, col, bonds = synth.sphere16(precision=precision)
    else:
        cfg, col, bonds = synth.poiseuille(precision=precision, L=(16, 12, 10))
    x, v, fl = synth.solvent(cfg, col, seed=11, frac_b=0.3)
    s = api.System.single(cfg, len(x), col, bonds, precision=precision)
    s.set_state(0, x, v, fl)
    s.step(3)
    L = cfg["L"]
    n_cells = L[0] * L[1] * (L[2] + (1 if cfg["walls"] else 0))
    return s, len(x), n_cells


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["sphere16", "walls"])
def test_noalloc_matches_observables_on_two_calls_in_a_row(lib, kind, precision):
    import torch
    s, n, n_cells = _system(kind, precision)
    assert n_cells <= api.RMPCD_NOALLOC_MAX_CELLS
    ref = s.observables(0)
    dev = torch.device("cuda")
    st = {"v": torch.empty((n, 3), dtype=torch.float64, device=dev),
          "flags": torch.empty(n, dtype=torch.uint8, device=dev),
          "cell": torch.empty(n, dtype=torch.int32, device=dev)}
    s.get_state(0, out=st)
    assert int(st["cell"].min()) >= 0 and int(st["cell"].max()) < n_cells
    vabs = float(st["v"].abs().sum(dim=0).max())
    # both sum in FP64, in different orders (atomics here): the tolerance of each path's parity tests
    tol = 1e-5 if precision == "mixed" else 1e-12
    out = torch.empty(8, dtype=torch.float64, device=dev)
    for call in range(2):
        out.fill_(float("nan"))
        api.observables_noalloc(st["cell"], st["v"], st["flags"], n_cells, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o)), (call, o)
        assert o[5] == ref["n_cells_used"], (call, o[5], ref["n_cells_used"])
        assert o[6] == ref["n_B"] and o[7] == ref["n_solvent"] == n, (call, o)
        assert abs(o[0] - ref["temperature"]) <= tol * ref["temperature"], (call, o[0], ref["temperature"])
        assert abs(o[4] - ref["kinetic"]) <= tol * ref["kinetic"], (call, o[4], ref["kinetic"])
        assert np.all(np.abs(o[1:4] - ref["momentum"]) <= tol * vabs), (call, o[1:4], ref["momentum"])
    s.close()


def test_binding_limit_matches_the_header():
    """api.RMPCD_NOALLOC_MAX_CELLS is a copy of the header's macro: keep them equal."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "rmpcd.h")).read()
    m = re.search(r"#define\s+RMPCD_NOALLOC_MAX_CELLS\s+(\d+)", hdr)
    assert m and int(m.group(1)) == api.RMPCD_NOALLOC_MAX_CELLS


def test_binding_rejects_bad_tensors_before_the_call():
    """The binding checks dtype, shape, layout and device before handing raw
    pointers to the library (no GPU needed: every case fails in Python)."""
    torch = pytest.importorskip("torch")
    n = 10
    ok = dict(cell=torch.zeros(n, dtype=torch.int32), v=torch.zeros(n, 3, dtype=torch.float64),
              flags=torch.zeros(n, dtype=torch.uint8), out=torch.zeros(8, dtype=torch.float64))
    bad = [
        ("v", torch.zeros(n, 3, dtype=torch.float32), "float64"),
        ("cell", torch.zeros(n, dtype=torch.int64), "int32"),
        ("flags", torch.zeros(n, dtype=torch.int32), "uint8"),
        ("out", torch.zeros(8, dtype=torch.float32), "float64"),
        ("v", torch.zeros(3, n, dtype=torch.float64).t(), "contiguous"),
        ("v", torch.zeros(n - 1, 3, dtype=torch.float64), "shape"),
        ("flags", torch.zeros(n - 1, dtype=torch.uint8), "entries"),
        ("out", torch.zeros(7, dtype=torch.float64), "8 doubles"),
        ("cell", torch.zeros(n, 1, dtype=torch.int32), "1-D"),
    ]
    for name, t, word in bad:
        args = dict(ok)
        args[name] = t
        with pytest.raises(ValueError, match=word):
            api.observables_noalloc(args["cell"], args["v"], args["flags"], 16, args["out"])
    # well-formed host tensors are still refused: the library takes device pointers
    with pytest.raises(ValueError, match="CUDA"):
        api.observables_noalloc(ok["cell"], ok["v"], ok["flags"], 16, ok["out"])
    with pytest.raises(ValueError, match="CUDA"):
        api.observables_noalloc(ok["cell"], ok["v"], None, 16, ok["out"])
