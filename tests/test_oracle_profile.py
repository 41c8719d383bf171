"""Pins of the oracle's slab profile (the flow profile, slab temperature and
species profile of §"Applications of RMPCDMD") against brute force with exact
rational arithmetic, conservation sums, hand-built slabs with closed-form
moments and the statistics of a Maxwell-Boltzmann solvent."""
import math
from fractions import Fraction

import numpy as np
import pytest


def _brute(L, x, v, fl, n_bins):
    """Per-particle loop with exact rationals: bin floor(x n / L), each term
    rounded half-to-even on its fixed-point grid (Python's round)."""
    n = [0] * n_bins
    nB = [0] * n_bins
    s1 = [[0, 0, 0] for _ in range(n_bins)]
    s2 = [[0, 0, 0] for _ in range(n_bins)]
    for i in range(len(x)):
        b = math.floor(Fraction(float(x[i])) * n_bins / L)
        b = min(max(b, 0), n_bins - 1)
        n[b] += 1
        nB[b] += int(fl[i]) & 1
        for k in range(3):
            q = Fraction(float(v[i, k]))
            s1[b][k] += round(q * 2 ** 32)
            s2[b][k] += round(Fraction(float(v[i, k]) * float(v[i, k])) * 2 ** 24)
    return n, nB, s1, s2


@pytest.mark.parametrize("axis,n_bins", [(0, 7), (1, 1), (2, 12)])
def test_profile_matches_exact_brute_force(orc, axis, n_bins):
    rng = np.random.default_rng(11 + axis)
    L = (9, 10, 12)
    x = rng.uniform(0.0, 1.0, (400, 3)) * np.asarray(L, float)
    x[:5, axis] = [0.0, L[axis], L[axis] - 1e-12, L[axis] * 0.5, 1e-300]   # edges and the wall position
    v = rng.normal(0.0, 1.3, (400, 3))
    v[0] = [0.5 * 2 ** -32, 1.5 * 2 ** -32, -0.5 * 2 ** -32]   # ties round to even
    fl = rng.integers(0, 4, 400).astype(np.uint8)
    p = orc.slab_profile(L[axis], x[:, axis], v, fl, n_bins)
    n, nB, s1, s2 = _brute(L[axis], x[:, axis], v, fl, n_bins)
    assert p["n"].tolist() == n
    assert p["n_B"].tolist() == nB
    assert np.array_equal(p["v_sum"], np.array(s1, float) * 2.0 ** -32)
    assert np.array_equal(p["v2_sum"], np.array(s2, float) * 2.0 ** -24)
    # the two particles at L and L - 1e-12 land in the last bin, 0 and 1e-300 in the first
    assert p["n"][-1] >= 2 and p["n"][0] >= 2


def test_profile_sums_are_the_totals(orc):
    """Summed over bins: N, N_B, total momentum and twice the kinetic energy,
    within the per-term rounding (N x half a grid step)."""
    rng = np.random.default_rng(3)
    N, L = 5000, 16
    x = rng.uniform(0, L, N)
    v = rng.normal(0.2, 1.0, (N, 3))
    fl = (rng.uniform(size=N) < 0.3).astype(np.uint8)
    p = orc.slab_profile(L, x, v, fl, 16)
    assert p["n"].sum() == N and p["n_B"].sum() == int(fl.sum())
    assert np.all(np.abs(p["v_sum"].sum(0) - v.sum(0)) <= N * 2.0 ** -33)
    assert np.all(np.abs(p["v2_sum"].sum(0) - (v * v).sum(0)) <= N * 2.0 ** -25)


def test_hand_built_slabs_give_closed_form_moments(orc):
    """Slab b holds 2m particles moving with u_b +- d_b along x and +- e along
    y: mean flow (u_b, 0, 0), temperature (2m (d_b^2 + e^2)) / (3 (2m - 1)).
    All values are dyadic, so every sum is exact."""
    L, nb, m = 8, 4, 5
    u = np.array([0.25, -0.5, 1.0, 0.125])
    d = np.array([0.5, 0.75, 0.25, 1.0])
    e = 0.375
    xs, vs = [], []
    for b in range(nb):
        for j in range(2 * m):
            s = 1.0 if j % 2 == 0 else -1.0
            xs.append(b * L / nb + (j + 0.5) * (L / nb) / (2 * m))
            vs.append([u[b] + s * d[b], -s * e, 0.0])
    p = orc.slab_profile(L, np.array(xs), np.array(vs), None, nb)
    f = orc.slab_fields(p)
    assert p["n"].tolist() == [2 * m] * nb
    assert np.array_equal(f["u"][:, 0], u) and np.array_equal(f["u"][:, 1:], np.zeros((nb, 2)))
    assert np.allclose(f["T"], 2 * m * (d ** 2 + e ** 2) / (3 * (2 * m - 1)), rtol=1e-15)
    assert np.all(f["c_B"] == 0.0)


def test_axis_selects_the_position_component(orc):
    """All particles share x_0 = 1.5 but spread along axis 2: binning axis 0
    puts them in one bin, axis 2 spreads them uniformly."""
    L = 6
    x = np.stack([np.full(600, 1.5), np.zeros(600), (np.arange(600) + 0.5) * L / 600], 1)
    v = np.zeros((600, 3))
    assert orc.slab_profile(L, x[:, 0], v, None, 6)["n"].tolist() == [0, 600, 0, 0, 0, 0]
    assert orc.slab_profile(L, x[:, 2], v, None, 6)["n"].tolist() == [100] * 6


def test_maxwell_slabs_recover_temperature_and_shear_flow(orc):
    """A Maxwell-Boltzmann solvent at kT 1.3 carrying the shear flow
    u_x = 0.05 (z - L/2): slab T within 5 standard errors of kT (SE of the
    sample variance estimate, sqrt(2/(3n)) kT) and slab mean flow within 5 SE
    of u_x at the slab's mean height."""
    rng = np.random.default_rng(7)
    N, L, nb, kT = 60000, 12, 12, 1.3
    z = rng.uniform(0, L, N)
    v = rng.normal(0.0, math.sqrt(kT), (N, 3))
    v[:, 0] += 0.05 * (z - L / 2)
    p = orc.slab_profile(L, z, v, None, nb)
    f = orc.slab_fields(p)
    zb = np.array([z[np.floor(z * nb / L).astype(int) == b].mean() for b in range(nb)])
    n = p["n"].astype(float)
    # the shear within a slab (width 1) adds (0.05^2 / 12) / 3 to T
    T_want = kT + 0.05 ** 2 / 12.0 / 3.0
    assert np.all(np.abs(f["T"] - T_want) < 5 * T_want * np.sqrt(2.0 / (3.0 * n)))
    assert np.all(np.abs(f["u"][:, 0] - 0.05 * (zb - L / 2)) < 5 * math.sqrt(kT) / np.sqrt(n))
