"""Pins of the oracle's counter-based generator and of the draws built on it."""
import os
import shutil
import subprocess
import sysconfig

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    """Published known-answer vectors of Philox4x32-10 (Salmon et al. SC'11)."""
    for ctr, key, want in _kat():
        got = orc.philox4x32_10(ctr, key)
        assert [int(a) for a in got] == want


def _torch_include():
    try:
        import torch
    except Exception:
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    return inc if os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) else None


def test_philox_matches_an_independent_implementation(orc, tmp_path):
    """Cross-check against the Philox4x32-10 that ships as a C++ header with
    PyTorch (compiled and called here, not copied)."""
    inc = _torch_include()
    gxx = shutil.which("g++")
    if inc is None or gxx is None:
        pytest.skip("PyTorch C++ headers or g++ not available")
    src = tmp_path / "ph.cpp"
    src.write_text(
        "#include <ATen/core/PhiloxRNGEngine.h>\n#include <cstdio>\n#include <cstdlib>\n"
        "int main(int argc, char** argv){ unsigned long long seed = strtoull(argv[1],0,10),"
        " sub = strtoull(argv[2],0,10), off = strtoull(argv[3],0,10);\n"
        " at::Philox4_32 e(seed, sub, off); for(int i=0;i<4;++i) printf(\"%u \", e()); return 0; }\n")
    exe = tmp_path / "ph"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("could not compile the PyTorch Philox header: " + r.stderr[-300:])
    rng = np.random.Generator(np.random.PCG64(7))
    for _ in range(40):
        seed = int(rng.integers(0, 2**63))
        sub = int(rng.integers(0, 2**63))
        off = int(rng.integers(0, 2**63))
        out = subprocess.run([str(exe), str(seed), str(sub), str(off)], capture_output=True,
                             text=True, check=True).stdout.split()
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert [int(a) for a in orc.philox4x32_10(ctr, key)] == [int(t) for t in out]


def test_grid_shift_is_uniform_on_24_bit_grid(orc):
    s = np.array([orc.grid_shift(12345, k) for k in range(4000)])
    assert s.min() >= 0.0 and s.max() < 1.0
    assert np.all(s * 2**24 == np.floor(s * 2**24))
    # mean 1/2, variance 1/12 per component, within 5 standard errors
    se_mean = np.sqrt(1 / 12 / len(s))
    assert np.all(np.abs(s.mean(0) - 0.5) < 5 * se_mean)
    assert np.all(np.abs(s.var(0) - 1 / 12) < 0.01)
    # different steps and seeds give different shifts
    assert not np.allclose(orc.grid_shift(1, 0), orc.grid_shift(1, 1))
    assert not np.allclose(orc.grid_shift(1, 0), orc.grid_shift(2, 0))


def test_rotation_axis_uniform_on_sphere(orc):
    n = np.array([orc.rotation_axis(99, 3, c) for c in range(20000)])
    norms = np.linalg.norm(n, axis=1)
    assert np.max(np.abs(norms - 1.0)) < 4e-16 * 4
    # isotropy: <n> = 0 and <n n^T> = I/3 (standard errors ~ 1/sqrt(3N))
    assert np.all(np.abs(n.mean(0)) < 5 / np.sqrt(3 * len(n)))
    cov = n.T @ n / len(n)
    assert np.allclose(cov, np.eye(3) / 3, atol=0.015)
    # the z component of a uniform point on the sphere is uniform on [-1, 1]
    from scipy import stats
    assert stats.kstest(n[:, 2], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3
