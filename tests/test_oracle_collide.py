"""Pins of the oracle's collision step (§1.4: SRD rule, MPC-AT) and of the
temperature estimator, against invariants and the SRD transport closed forms.

The closed forms for the self-diffusion coefficient and the kinematic
viscosity of SRD with random shift are the standard kinetic-theory results
(Ihle & Kroll 2001; Kikuchi et al. 2003; Ripoll et al. 2005), which the paper
cites for the method but does not print; they hold to a few percent at the
mean free paths used here."""
import math

import numpy as np
from scipy import stats

from paper_1608_04904_gb300 import synth


def _sorted_system(orc, cfg, n=None, seed=21, **kw):
    x, v, fl = synth.solvent(cfg, n=n, seed=seed, **kw)
    s = orc.OracleSystem(cfg, x, v, fl)
    s.shift_and_sort()
    return s


def _cell_sums(s, v):
    mom = np.zeros((s.ncells, 3))
    ke = np.zeros(s.ncells)
    np.add.at(mom, s.key, v)
    np.add.at(ke, s.key, (v * v).sum(1))
    return mom, ke


def test_srd_conserves_cell_momentum_and_energy(orc):
    cfg = synth.base_config(L=(8, 8, 8), alpha=math.radians(130.0))
    s = _sorted_system(orc, cfg)
    m0, e0 = _cell_sums(s, s.v)
    v_before = s.v.copy()
    s.collide()
    m1, e1 = _cell_sums(s, s.v)
    assert np.max(np.abs(m1 - m0)) < 1e-13 * max(1.0, np.abs(m0).max())
    assert np.max(np.abs(e1 - e0)) < 1e-13 * max(1.0, e0.max())
    # something did change in every cell with >= 2 particles
    moved = np.zeros(s.ncells, dtype=bool)
    np.logical_or.at(moved, s.key, np.any(s.v != v_before, axis=1))
    assert np.all(moved[s.count >= 2])
    # singly occupied cells are untouched
    single = s.count[s.key] == 1
    assert np.array_equal(s.v[single], v_before[single])


def test_srd_rotates_relative_velocity_by_plus_alpha(orc):
    alpha = math.radians(130.0)
    cfg = synth.base_config(L=(4, 4, 4), alpha=alpha)
    s = _sorted_system(orc, cfg, n=600)
    v0 = s.v.copy()
    s.collide()
    checked = 0
    for c in range(s.ncells):
        N = s.count[c]
        if N < 2:
            continue
        sl = slice(s.start[c], s.start[c] + N)
        vcm = v0[sl].mean(0)
        u0 = v0[sl] - vcm
        u1 = s.v[sl] - vcm
        n = orc.rotation_axis(cfg["seed"], 0, c)
        for a, b in zip(u0, u1):
            # component along the axis is kept
            assert abs(a @ n - b @ n) < 1e-12
            pa, pb = a - (a @ n) * n, b - (b @ n) * n
            if np.linalg.norm(pa) < 1e-6:
                continue
            cosang = pa @ pb / (np.linalg.norm(pa) * np.linalg.norm(pb))
            sinang = np.cross(pa, pb) @ n / (np.linalg.norm(pa) * np.linalg.norm(pb))
            # right-handed rotation by +alpha about n
            assert abs(cosang - math.cos(alpha)) < 1e-10
            assert abs(sinang - math.sin(alpha)) < 1e-10
            checked += 1
    assert checked > 300


def test_zero_angle_is_identity(orc):
    cfg = synth.base_config(L=(6, 6, 6), alpha=0.0)
    s = _sorted_system(orc, cfg)
    v0 = s.v.copy()
    s.collide()
    assert np.max(np.abs(s.v - v0)) < 1e-15 * 8


def test_temperature_estimator_unbiased_at_equilibrium(orc):
    for kT in (1.0, 1.0 / 3.0):
        cfg = synth.base_config(L=(16, 16, 16), kT=kT)
        s = _sorted_system(orc, cfg, seed=5)
        T = s.temperature()
        # relative standard error ~ sqrt(2 / (3 sum (N_xi - 1))) over all cells
        se = kT * math.sqrt(2.0 / (3.0 * (s.count[s.count >= 2] - 1).sum()))
        assert abs(T - kT) < 4 * se


def test_relaxes_to_maxwell_boltzmann(orc):
    """Start every particle at speed sqrt(3 kT) in a random direction; after
    collisions the velocity components must be Gaussian at kT (§1.2, the
    equilibrium velocity distribution check)."""
    cfg = synth.base_config(L=(16, 16, 16), kT=1.0, alpha=math.radians(130.0), tau=0.5)
    x, v, fl = synth.solvent(cfg, seed=8)
    rng = np.random.Generator(np.random.PCG64(9))
    d = rng.standard_normal(v.shape)
    d /= np.linalg.norm(d, axis=1)[:, None]
    v = d * math.sqrt(3.0)
    v -= v.mean(0)
    s = orc.OracleSystem(cfg, x, v, fl)
    assert stats.kstest(s.v[:, 0], stats.norm(scale=1.0).cdf).pvalue < 1e-6
    s.step(20)
    for k in range(3):
        assert stats.kstest(s.v[:, k], stats.norm(scale=1.0).cdf).pvalue > 1e-4
    assert abs((s.v ** 2).sum(1).mean() - 3.0) < 3e-2


def _d_closed(kT, tau, M, alpha):
    return kT * tau / 2.0 * (3.0 * M / ((M - 1.0 + math.exp(-M)) * (1.0 - math.cos(alpha))) - 1.0)


def _nu_closed(kT, tau, M, alpha):
    g = M - 1.0 + math.exp(-M)
    nu_kin = kT * tau / 2.0 * (5.0 * M / (g * (2.0 - math.cos(alpha) - math.cos(2 * alpha))) - 1.0)
    nu_col = (1.0 - math.cos(alpha)) / (18.0 * tau) * g / M
    return nu_kin + nu_col


def test_closed_form_values_used_elsewhere():
    assert abs(_d_closed(1.0, 0.5, 10, math.radians(130)) - 0.2573) < 5e-4
    assert abs(_nu_closed(1.0, 0.5, 10, math.radians(130)) - 0.4074) < 5e-4
    assert abs(_nu_closed(1.0, 1.0, 10, math.radians(130)) - 0.5684) < 5e-4


def test_self_diffusion_matches_closed_form(orc):
    alpha, tau, kT = math.radians(130.0), 0.5, 1.0
    cfg = synth.base_config(L=(16, 16, 16), alpha=alpha, tau=tau, kT=kT, seed=31)
    x, v, fl = synth.solvent(cfg, seed=31)
    s = orc.OracleSystem(cfg, x, v, fl)
    s.step(5)
    disp = np.zeros((s.n, 3))
    msd = []
    for k in range(60):
        order = np.argsort(s.id)
        disp += s.v[order] * tau          # free flight displacement of the next interval
        s.step(1)
        msd.append((disp ** 2).sum(1).mean())
    k0, k1 = 20, 60
    D = (msd[k1 - 1] - msd[k0 - 1]) / (6.0 * (k1 - k0) * tau)
    Dth = _d_closed(kT, tau, 10, alpha)
    assert abs(D - Dth) / Dth < 0.05, (D, Dth)


def test_shear_wave_decay_matches_closed_form_viscosity(orc):
    alpha, tau, kT = math.radians(130.0), 0.5, 1.0
    L = 16
    cfg = synth.base_config(L=(L, L, L), alpha=alpha, tau=tau, kT=kT, seed=41)
    x, v, fl = synth.solvent(cfg, seed=41)
    k = 2 * math.pi / L
    v[:, 0] += 0.5 * np.sin(k * x[:, 2])
    s = orc.OracleSystem(cfg, x, v, fl)
    amp = []
    for _ in range(40):
        amp.append(2.0 * np.mean(s.v[:, 0] * np.sin(k * s.x[:, 2])))
        s.step(1)
    t = np.arange(len(amp)) * tau
    rate = -np.polyfit(t[2:], np.log(amp[2:]), 1)[0]
    nu = rate / k ** 2
    nuth = _nu_closed(kT, tau, 10, alpha)
    assert abs(nu - nuth) / nuth < 0.06, (nu, nuth)


def test_mpc_at_slab_thermalises_and_conserves_cell_momentum(orc):
    cfg = synth.base_config(L=(8, 8, 8), kT=1.0, slabs=[(0.0, 8.0, 2.0)])
    s = _sorted_system(orc, cfg, seed=3)
    m0, _ = _cell_sums(s, s.v)
    s.collide()
    m1, _ = _cell_sums(s, s.v)
    assert np.max(np.abs(m1 - m0)) < 1e-12
    T = s.temperature()
    se = 2.0 * math.sqrt(2.0 / (3.0 * (s.count[s.count >= 2] - 1).sum()))
    assert abs(T - 2.0) < 5 * se


def test_mpc_at_slabs_drive_a_linear_temperature_profile(orc):
    """Two MPC-AT slabs (kT 1.2 on [0, 2), 0.8 on [16, 18)) in a periodic
    32-cell column: in steady state the slab temperatures hold inside the
    slabs, the profile between them is linear (Fourier's law with a constant
    conductivity) with a gradient close to (0.8 - 1.2) / 14 per cell (slightly
    less: the slabs' edges take part of the drop), and the two halves of the
    periodic column mirror each other about the slabs' mean centres."""
    cfg = synth.base_config(L=(32, 8, 8), alpha=np.radians(130.0), tau=0.5, kT=1.0, seed=41,
                            slabs=[(0.0, 2.0, 1.2), (16.0, 18.0, 0.8)])
    x, v, fl = synth.solvent(cfg, seed=42)
    o = orc.OracleSystem(cfg, x, v, fl)
    o.step(200)
    T = np.zeros(32)
    for _ in range(400):
        o.step(1)
        T += orc.slab_fields(orc.slab_profile(32, o.x[:, 0], o.v, o.flags, 32))["T"]
    T /= 400
    assert abs(T[1] - 1.2) < 0.02 and abs(T[17] - 0.8) < 0.02
    b = np.arange(4, 15)
    slope, icpt = np.polyfit(b + 0.5, T[b], 1)
    assert -0.4 / 14 * 1.15 < slope < -0.4 / 14 * 0.75, slope
    assert np.abs(T[b] - (slope * (b + 0.5) + icpt)).max() < 0.015
    # the slabs are columns of the shifted grid, [x0 + s, x1 + s) with s
    # uniform in [0, 1): centred at 1.5 and 17.5, so bin b mirrors bin 34 - b
    assert np.abs(T[b] - T[34 - b]).max() < 0.03
