"""Pins of the oracle's colloid-solvent dynamics (§1.1 velocity Verlet, §1.4
WCA potential, Verlet-list radius, exact RATTLE for the dimer; §1.5 catalytic
A->B conversion) against derivatives, brute force and conservation laws."""
import math

import numpy as np
import pytest

from paper_1608_04904_gb300 import synth


def test_wca_force_is_minus_gradient_of_energy(orc):
    sigma, eps = 2.0, 1.3
    rc = 2.0 ** (1 / 6) * sigma
    rng = np.random.Generator(np.random.PCG64(1))
    for r in np.linspace(0.85 * sigma, 0.999 * rc, 25):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        h = 1e-6
        hit, f, _ = orc.wca_force(r * u, sigma, eps)
        assert hit
        _, _, ep = orc.wca_force((r + h) * u, sigma, eps)
        _, _, em = orc.wca_force((r - h) * u, sigma, eps)
        dvdr = (ep - em) / (2 * h)
        assert np.allclose(f, -dvdr * u, rtol=1e-6, atol=1e-7)
    # energy and force vanish at the cut-off, and nothing acts beyond it
    hit, f, e = orc.wca_force(np.array([rc * (1 - 1e-9), 0, 0]), sigma, eps)
    assert hit and abs(e) < 1e-8 and np.linalg.norm(f) < 1e-6
    hit, f, e = orc.wca_force(np.array([0, rc * (1 + 1e-12), 0]), sigma, eps)
    assert not hit and e == 0 and not f.any()
    # the minimum of the full 12-6 potential is at 2^(1/6) sigma with depth -eps,
    # so the shifted WCA energy goes from eps at the minimum... to 0 at r_c
    _, _, e_mid = orc.wca_force(np.array([sigma, 0, 0]), sigma, eps)
    assert abs(e_mid - eps) < 1e-12   # V(sigma) = 4 eps (1 - 1 + 1/4) = eps


def test_colloid_force_equals_pair_sum(orc):
    """Summed colloid force equals minus the sum of brute-force pair forces."""
    cfg, col, _ = synth.dimer32(precision="fp64", L=12)
    cols = synth.colloid_arrays(col)
    x, v, fl = synth.solvent(cfg, col, n=3000, seed=4, frac_b=0.4, exclude_factor=0.8)
    f, F = orc.forces(cfg, x, fl, cols)
    L = np.asarray(cfg["L"], float)
    Fb = np.zeros((2, 3))
    fb = np.zeros_like(x)
    for i in range(len(x)):
        for j in range(2):
            d = x[i] - cols["x"][j]
            d -= L * np.round(d / L)
            eps = cols["eps_B"][j] if fl[i] & 1 else cols["eps_A"][j]
            hit, fij, _ = orc.wca_force(d, cols["sigma"][j], eps)
            if hit:
                fb[i] += fij
                Fb[j] -= fij
    assert np.allclose(f, fb, rtol=1e-14, atol=1e-14)
    assert np.allclose(F, Fb, rtol=1e-9, atol=1e-9)


def _dimer_system(orc, L=12, seed=2, **kw):
    cfg, col, bonds = synth.dimer32(precision="fp64", L=L)
    cfg.update(kw)
    x, v, fl = synth.solvent(cfg, col, seed=seed)
    return orc.OracleSystem(cfg, x, v, fl, colloids=synth.colloid_arrays(col), bonds=bonds)


def test_near_far_split_equals_substepping_everything(orc):
    a = _dimer_system(orc)
    b = _dimer_system(orc)
    a.interval(all_substep=False)
    b.interval(all_substep=True)
    near = a.near.astype(bool)
    assert 0 < near.sum() < a.n // 4
    assert np.array_equal(a.flags, b.flags)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.V, b.V)
    assert np.array_equal(a.x[near], b.x[near]) and np.array_equal(a.v[near], b.v[near])
    assert np.array_equal(a.v[~near], b.v[~near])
    # far particles: one flight over tau versus n_md flights of tau / n_md
    assert np.max(np.abs(a.x[~near] - b.x[~near])) < 1e-12


def test_nve_conserves_momentum_and_energy(orc):
    """No thermostat, walls or reactions: total momentum and energy conserved
    (the paper's continuous-integration check, §1.2)."""
    cfg, col, _ = synth.sphere16()
    cfg["L"] = (12, 12, 12)
    col[0]["x"] = (6.0, 6.0, 6.0)
    col[0]["v"] = (0.05, -0.02, 0.01)
    x, v, fl = synth.solvent(cfg, col, seed=6)
    s = orc.OracleSystem(cfg, x, v, fl, colloids=synth.colloid_arrays(col))
    p0 = s.momentum()
    e0 = s.kinetic_energy() + s.potential_energy()
    for _ in range(4):
        s.step(1)
        p1 = s.momentum()
        e1 = s.kinetic_energy() + s.potential_energy()
        assert np.max(np.abs(p1 - p0)) < 1e-8
        assert abs(e1 - e0) / e0 < 2e-5


def test_dimer_bond_is_rigid(orc):
    s = _dimer_system(orc)
    for _ in range(3):
        s.step(1)
        r = s.X[0] - s.X[1]
        assert abs(np.linalg.norm(r) - 4.5) < 1e-12
        assert abs((s.V[0] - s.V[1]) @ r) < 1e-12


def test_momentum_conserved_with_dimer(orc):
    s = _dimer_system(orc, bulk_rate=0.0)
    s.V[0] = [0.03, 0.0, 0.01]
    p0 = s.momentum()
    s.step(3)
    assert np.max(np.abs(s.momentum() - p0)) < 1e-8


def _probe(orc, cat_prob=1.0, tau=0.5, n_md=50):
    cfg, col, _ = synth.dimer32(precision="fp64", L=16)
    cfg.update(cat_prob=cat_prob, tau=tau, n_md=n_md)
    cols = synth.colloid_arrays(col)
    C = cols["x"][0]
    N = cols["x"][1]
    x = np.array([C + [0, 2.0, 0],      # A inside C's range, moving out
                  C + [0, 0, 3.0],      # A outside, moving away: untouched
                  N + [0, 2.0, 0],      # A inside the inert sphere, moving out: stays A
                  C + [0, -2.0, 0],     # B inside C moving out: stays B, never tagged
                  C + [0, 0, -2.1],     # tagged A at rest inside C's range
                  C + [-2.1, 0, 0.3]])  # untagged A at rest inside C's range
    v = np.array([[0, 3.0, 0], [0, 0, 1.0], [0, 3.0, 0], [0, -3.0, 0], [0, 0, 0], [0, 0, 0]])
    fl = np.array([0, 0, 0, 1, 2, 0], np.uint8)
    s = orc.OracleSystem(cfg, x, v, fl, colloids=cols, bonds=[(0, 1, 4.5)])
    s.interval()
    return s


def test_catalytic_conversion_on_leaving_c(orc):
    # over tau = 0.5 the WCA force expels the particles at rest too: every A
    # that was inside C's range has left it and converted
    s = _probe(orc)
    assert list(s.flags) == [1, 0, 0, 1, 1, 1]
    assert s.near.all()


def test_catalytic_tag_while_inside(orc):
    # over a short interval nobody leaves C's range: inside A particles carry
    # the tag, nothing converts
    s = _probe(orc, tau=0.02, n_md=2)
    assert list(s.flags) == [2, 0, 0, 1, 2, 2]


def test_catalytic_conversion_probability_zero(orc):
    s = _probe(orc, cat_prob=0.0)
    assert list(s.flags) == [0, 0, 0, 1, 0, 0]


def test_skin_violation_is_reported(orc):
    s = _dimer_system(orc)
    s.V[:] = [[2.0, 0, 0], [2.0, 0, 0]]
    with pytest.raises(orc.SkinError):
        s.interval()


def test_conversion_count_matches_tag_bookkeeping(orc):
    """With p = 1 every tagged A that ends outside all catalytic ranges is B."""
    s = _dimer_system(orc, L=16, bulk_rate=0.0)
    nb0 = int((s.flags & 1).sum())
    for _ in range(4):
        s.step(1)
    nb = int((s.flags & 1).sum())
    assert nb > nb0
    # tagged particles are A and inside C's range
    tagged = (s.flags & 2) != 0
    assert not np.any(tagged & ((s.flags & 1) != 0))
    L = np.asarray(s.cfg["L"], float)
    d = s.x[tagged] - np.mod(s.X[0], L)
    d -= L * np.round(d / L)
    assert np.all(np.linalg.norm(d, axis=1) < 2 ** (1 / 6) * 2.0)


def test_colloid_lj_force_is_minus_gradient_of_the_shifted_energy(orc):
    """Four spheres with colloid-colloid LJ (eps 1, sigma 3, cut 7.5): the
    force on each sphere is minus the central-difference gradient of the
    potential energy (energy shifted to zero at the cut); pairs beyond the cut
    and bonded pairs add nothing."""
    cfg = synth.base_config(L=(30, 30, 30), cc_lj=(1.0, 3.0, 7.5), seed=3)
    X = np.array([[10.0, 10.0, 10.0], [13.6, 10.4, 9.8], [11.2, 14.1, 10.9], [24.0, 24.0, 24.0]])
    col = [dict(x=tuple(p), v=(0.0, 0.0, 0.0), mass=100.0, sigma=1.0, eps_A=1.0, eps_B=1.0, catalytic=0)
           for p in X]
    F = orc.cc_forces(cfg, X)
    assert np.all(F[3] == 0.0)                       # sphere 3 is beyond every cut
    assert np.allclose(F.sum(0), 0.0, atol=1e-9)

    def energy(Xs, bonds=()):
        c = [dict(cc, x=tuple(p)) for cc, p in zip(col, Xs)]
        o = orc.OracleSystem(cfg, np.zeros((0, 3)), np.zeros((0, 3)), colloids=synth.colloid_arrays(c),
                             bonds=list(bonds))
        return o.potential_energy()

    h = 1e-5
    for j in range(3):
        for k in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[j, k] += h
            Xm[j, k] -= h
            g = (energy(Xp) - energy(Xm)) / (2 * h)
            assert abs(F[j, k] + g) < 1e-6 * max(1.0, abs(g)), (j, k, F[j, k], -g)
    # shifted: a pair just inside the cut has (almost) zero energy
    X2 = np.array([[10.0, 10.0, 10.0], [17.499, 10.0, 10.0]])
    assert abs(energy(X2)) < 1e-3 and np.abs(orc.cc_forces(cfg, X2)).max() < 0.02
    # a bonded pair is excluded
    Fb = orc.cc_forces(cfg, X, bonds=[(0, 1, 3.7)])
    F01 = orc.cc_forces(cfg, X[:2])
    assert np.allclose(Fb[:2], F[:2] - F01, atol=1e-9)
