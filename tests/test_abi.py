"""CPU checks of the C ABI: the library loads, exports what include/rmpcd.h
declares, and rejects invalid parameters before touching the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def api():
    from paper_1608_04904_gb300 import api, build
    build.build()
    return api


def _declared():
    src = open(os.path.join(ROOT, "include", "rmpcd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rmpcd_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(api):
    lib = api.load()
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(api.EXPORTS) == names


def test_struct_layouts_match_header(api, tmp_path):
    """Every field offset and struct size of the ctypes mirror equals what a C
    compiler makes of include/rmpcd.h."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    structs = {"rmpcd_params": api.Params, "rmpcd_colloid": api.Colloid, "rmpcd_bond": api.Bond,
               "rmpcd_obs": api.Obs, "rmpcd_timers": api.Timers, "rmpcd_body": api.Body, "rmpcd_bead": api.Bead,
               "rmpcd_profile_bin": api.ProfileBin, "rmpcd_net_bead": api.NetBead}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rmpcd.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def _create(api, params, colloids=None, bonds=None, cap=64, precision=1, n=1):
    lib = api.load()
    h = C.c_void_p()
    st = lib.rmpcd_create(C.byref(h), precision, n, params, colloids, bonds, cap, None)
    return st, lib.rmpcd_last_error(None).decode()


def _params(api, **kw):
    from paper_1608_04904_gb300 import synth
    cfg = synth.base_config(**kw)
    return api.make_params(cfg, 100)


@pytest.mark.parametrize("field,value,msg", [
    ("L", (1, 16, 16), "L[0]"),
    ("L", (16, 16, 2000), "L[2]"),
    ("n_md", 0, "n_md"),
    ("tau", 0.0, "tau"),
    ("cat_prob", 1.5, "cat_prob"),
    ("skin", -1.0, "skin"),
])
def test_invalid_parameters_are_rejected(api, field, value, msg):
    p = _params(api, **{field: value})
    st, err = _create(api, p)
    assert st == 1 and msg in err


def test_invalid_bucket_cap_and_precision(api):
    p = _params(api)
    st, err = _create(api, p, cap=-1)   # 0 is the automatic width
    assert st == 1 and "bucket_cap" in err
    st, err = _create(api, p, cap=100000)
    assert st == 1 and "bucket_cap" in err
    st, err = _create(api, p, precision=7)
    assert st == 1 and "precision" in err


def test_walls_need_no_z_force_and_no_colloids(api):
    p = _params(api, walls=1, rho_wall=10, g=(0.0, 0.0, 0.01))
    st, err = _create(api, p)
    assert st == 1 and "g[2]" in err
    p = _params(api, walls=1, rho_wall=10)
    p.n_colloids = 1
    col = (api.Colloid * 1)()
    col[0].mass, col[0].sigma = 1.0, 1.0
    st, err = _create(api, p, colloids=col)
    assert st == 1 and "walls" in err


def test_bad_bond_is_rejected(api):
    p = _params(api)
    p.n_colloids = 2
    p.n_bonds = 1
    col = (api.Colloid * 2)()
    for c in col:
        c.mass, c.sigma = 1.0, 1.0
    b = (api.Bond * 1)()
    b[0].a, b[0].b, b[0].d = 0, 0, 1.0
    st, err = _create(api, p, colloids=col, bonds=b)
    assert st == 1 and "bond" in err


def test_null_arguments(api):
    lib = api.load()
    assert lib.rmpcd_step(None, 1) == 1
    assert lib.rmpcd_sync(None) == 1
    lib.rmpcd_destroy(None)
    h = C.c_void_p()
    assert lib.rmpcd_create(C.byref(h), 1, 0, None, None, None, 64, None) == 1


def _dimer_replica(**kw):
    from paper_1608_04904_gb300 import synth
    cfg, col, bonds = synth.dimer32(precision="mixed", **kw)
    return dict(cfg=cfg, n=int(cfg["rho"] * 32 ** 3), colloids=col, bonds=bonds)


def test_workspace_size_counts_the_buffers_without_a_gpu(api):
    """rmpcd_workspace_size makes no CUDA call.  Its answer grows with the
    bucket width by exactly the two arrays of cell rows (cells x width x one
    record each -- 32 bytes mixed, 64 FP64 --, rounded to 256), with the
    particle count by at least the two record buffers, and the FP64 records
    (64 B) need more than the mixed ones (32 B)."""
    rep = _dimer_replica()
    cells = 32 ** 3
    r256 = lambda b: (b + 255) // 256 * 256
    a = api.workspace_size([rep], "mixed", 48)
    b = api.workspace_size([rep], "mixed", 64)
    assert b - a == 2 * (r256(cells * 64 * 32) - r256(cells * 48 * 32))
    a64 = api.workspace_size([rep], "fp64", 48)
    assert api.workspace_size([rep], "fp64", 64) - a64 == 2 * (r256(cells * 64 * 64) - r256(cells * 48 * 64))
    big = dict(rep, n=rep["n"] + 8192)
    assert api.workspace_size([big], "mixed", 48) - a >= 2 * 32 * 8192
    assert api.workspace_size([rep], "fp64", 48) - a >= 2 * 32 * rep["n"]
    # two replicas need the sum of the per-replica buffers, give or take the
    # per-system ones
    two = api.workspace_size([rep, rep], "mixed", 48)
    assert a < two < 2 * a
    # bucket_cap 0: the autotuned width, which at density 10 is 32..64
    auto = api.workspace_size([rep], "mixed", 0)
    assert api.workspace_size([rep], "mixed", 32) <= auto <= b


def test_workspace_size_rejects_what_create_rejects(api):
    from paper_1608_04904_gb300 import synth
    rep = _dimer_replica()
    with pytest.raises(api.RmpcdError):
        api.workspace_size([dict(rep, cfg=dict(rep["cfg"], L=(1, 32, 32)))], "mixed", 48)
    with pytest.raises(api.RmpcdError):
        api.workspace_size([rep], "mixed", 100000)
    lib = api.load()
    p = api.make_params(synth.base_config(), 100)
    assert lib.rmpcd_workspace_size(1, 1, p, None, None, 64, None) == 1


def test_reservoir_columns_outside_the_box_are_rejected(api):
    """rmpcd_workspace_size validates like rmpcd_create, without a GPU."""
    from paper_1608_04904_gb300 import synth
    cfg = synth.base_config(L=(8, 16, 6), reservoirs=((0, 2), (14, 17)))
    with pytest.raises(api.RmpcdError) as e:
        api.workspace_size([dict(cfg=cfg, n=100)], "fp64", 64)
    assert e.value.code == "EINVAL"
    ok = synth.base_config(L=(8, 16, 6), reservoirs=((0, 2), (14, 16)))
    assert api.workspace_size([dict(cfg=ok, n=100)], "fp64", 64) > 0
