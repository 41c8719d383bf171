"""Pins of the oracle's free flight with body force and bounce-back walls,
virtual wall particles (§1.4) and the bulk RMPCD reaction (§1.1, Appendix A)."""
import math

import numpy as np

from paper_1608_04904_gb300 import synth


def test_free_flight_with_body_force_is_ballistic(orc):
    cfg = synth.base_config(L=(10, 10, 10), g=(0.01, -0.02, 0.005), tau=0.7)
    x = np.array([[1.0, 2.0, 3.0], [9.5, 0.2, 5.0]])
    v = np.array([[0.3, -0.1, 0.2], [1.0, -0.5, 0.0]])
    s = orc.OracleSystem(cfg, x, v)
    s.interval()
    g = np.asarray(cfg["g"])
    t = cfg["tau"]
    want = np.mod(x + v * t + 0.5 * g * t * t, 10.0)
    assert np.allclose(s.x, want, atol=1e-14)
    assert np.allclose(s.v, v + g * t, atol=1e-15)


def test_bounce_back_reverses_velocity_at_wall(orc):
    cfg = synth.base_config(L=(8, 8, 6), walls=1, rho_wall=10, tau=1.0)
    x = np.array([[2.0, 3.0, 0.3], [4.0, 4.0, 5.8], [1.0, 1.0, 3.0]])
    v = np.array([[0.5, 0.2, -1.0], [0.1, -0.3, 0.5], [0.2, 0.1, 0.4]])
    s = orc.OracleSystem(cfg, x, v)
    s.interval()
    # particle 0 hits z = 0 at t = 0.3, then flies 0.7 with -v
    assert np.allclose(s.x[0], [2.0 + 0.5 * 0.3 - 0.5 * 0.7, 3.0 + 0.2 * 0.3 - 0.2 * 0.7, 0.7], atol=1e-14)
    assert np.allclose(s.v[0], -v[0])
    # particle 1 hits z = 6 at t = 0.4, then flies 0.6 with -v
    assert np.allclose(s.x[1], [4.0 + 0.1 * 0.4 - 0.1 * 0.6, 4.0 - 0.3 * 0.4 + 0.3 * 0.6, 6.0 - 0.5 * 0.6],
                       atol=1e-14)
    assert np.allclose(s.v[1], -v[1])
    # particle 2 does not reach a wall
    assert np.allclose(s.x[2], x[2] + v[2]) and np.array_equal(s.v[2], v[2])


def test_poiseuille_profile_matches_closed_form_viscosity(orc):
    """Stick walls (bounce-back + virtual particles) and a body force give the
    parabolic profile v_x(z) = g z (H - z) / (2 nu) (§1.5 ``poiseuille_flow``),
    nu from the SRD closed form."""
    H = 12
    g = 0.005
    alpha, tau, kT = math.radians(130.0), 1.0, 1.0
    cfg = synth.base_config(L=(10, 10, H), walls=1, rho_wall=10, g=(g, 0.0, 0.0), alpha=alpha, tau=tau,
                            kT=kT, seed=17)
    x, v, fl = synth.solvent(cfg, seed=17)
    s = orc.OracleSystem(cfg, x, v, fl)
    s.step(150)
    nb = 12
    acc = np.zeros(nb)
    cnt = np.zeros(nb)
    temps = []
    for _ in range(250):
        s.step(1)
        temps.append(s.temperature())
        b = np.minimum((s.x[:, 2] / H * nb).astype(int), nb - 1)
        acc += np.bincount(b, weights=s.v[:, 0], minlength=nb)
        cnt += np.bincount(b, minlength=nb)
    prof = acc / cnt
    z = (np.arange(nb) + 0.5) * H / nb
    shape = z * (H - z)
    a = (prof @ shape) / (shape @ shape)       # least-squares amplitude of z (H - z)
    # no thermostat: viscous heating warms the fluid slowly, so the closed form
    # is taken at the measured mean temperature of the averaging window
    kTm = float(np.mean(temps))
    assert 1.0 < kTm < 1.2
    M = 10.0
    gm = M - 1.0 + math.exp(-M)
    nu = (kTm * tau / 2.0 * (5.0 * M / (gm * (2.0 - math.cos(alpha) - math.cos(2 * alpha))) - 1.0)
          + (1.0 - math.cos(alpha)) / (18.0 * tau) * gm / M)
    assert abs(a - g / (2.0 * nu)) / (g / (2.0 * nu)) < 0.06, (a, g / (2 * nu))
    # the residual from the parabola is small (no plug flow, no slip offset)
    assert np.max(np.abs(prof - a * shape)) < 0.1 * a * shape.max()


def test_virtual_particles_pull_wall_cells_toward_rest(orc):
    """A wall cell with N < rho_wall real particles gets rho_wall - N virtual
    ones whose summed momentum has zero mean, so E[v_cm] = (N / rho_wall) V for
    real particles all moving with V.  After the rotation about a uniform axis
    (E[R] = (1 + 2 cos a) / 3) the real particles' mean velocity averages to
    v_cm + (1 + 2 cos a) / 3 (V - v_cm)."""
    alpha = math.radians(130.0)
    cfg = synth.base_config(L=(4, 4, 4), walls=1, rho_wall=10, alpha=alpha, kT=1.0)
    x = np.array([[1.50, 2.50, 0.001], [1.505, 2.505, 0.002], [1.495, 2.495, 0.003]])
    v = np.tile([1.0, 0.0, 0.0], (3, 1))
    means = []
    for step in range(600):
        s = orc.OracleSystem(cfg, x, v, step=step)
        s.shift_and_sort()
        if s.count.max() != 3 or s.key[0] // 16 != 0:
            continue
        s.collide()
        means.append(s.v[:, 0].mean())
    means = np.asarray(means)
    assert len(means) > 500
    f = 3.0 / 10.0
    want = f + (1.0 + 2.0 * math.cos(alpha)) / 3.0 * (1.0 - f)
    se = means.std() / math.sqrt(len(means))
    assert abs(means.mean() - want) < 4 * se, (means.mean(), want, se)
    # without virtual particles (interior cell) momentum is conserved exactly
    x2 = x.copy()
    x2[:, 2] += 2.0
    s = orc.OracleSystem(cfg, x2, v)
    s.shift_and_sort()
    s.collide()
    assert abs(s.v[:, 0].mean() - 1.0) < 1e-14


def test_single_particle_wall_cell_collides_with_virtual_partners(orc):
    """A wall cell holding ONE real particle still gets rho_wall - 1 virtual
    partners (§1.4, virtual particles after Lamura et al. 2001): v_cm = (V +
    P_v) / rho_wall differs from V, so the collision is not the identity.  With
    f = 1 / rho_wall, E[v_cm] = f V and E[R] = (1 + 2 cos a) / 3, so the
    particle's velocity after the collision averages f V + (1 + 2 cos a) / 3
    (1 - f) V.  A rule that skips cells with N < 2 leaves it at V."""
    alpha = math.radians(130.0)
    rho_wall = 10
    cfg = synth.base_config(L=(4, 4, 4), walls=1, rho_wall=rho_wall, alpha=alpha, kT=1.0)
    x = np.array([[1.50, 2.50, 0.001]])
    V = np.array([[1.0, -0.5, 0.25]])
    got = []
    for step in range(800):
        s = orc.OracleSystem(cfg, x, V, step=step)
        s.shift_and_sort()
        if s.key[0] // 16 != 0:   # the particle must sit in the bottom wall layer
            continue
        s.collide()
        got.append(s.v[0].copy())
    got = np.asarray(got)
    assert len(got) > 700
    f = 1.0 / rho_wall
    want = (f + (1.0 + 2.0 * math.cos(alpha)) / 3.0 * (1.0 - f)) * V[0]
    se = got.std(axis=0) / math.sqrt(len(got))
    assert np.all(np.abs(got.mean(axis=0) - want) < 4 * se), (got.mean(axis=0), want, se)
    # every sample moved: the collision is never the identity here
    assert np.all(np.abs(got - V).sum(axis=1) > 0)
    # the same particle away from the walls is a lone particle: unchanged
    s = orc.OracleSystem(cfg, x + [0.0, 0.0, 2.0], V)
    s.shift_and_sort()
    s.collide()
    assert np.array_equal(s.v, V)


def _cells(orc, cfg, nb_frac, seed):
    x, v, fl = synth.solvent(cfg, seed=seed, frac_b=nb_frac)
    s = orc.OracleSystem(cfg, x, v, fl)
    s.shift_and_sort()
    return s


def test_bulk_reaction_certain_converts_one_b_per_cell(orc):
    cfg = synth.base_config(L=(6, 6, 6), bulk_rate=1e6)
    s = _cells(orc, cfg, 0.5, 3)
    nb0 = np.bincount(s.key, weights=(s.flags & 1), minlength=s.ncells)
    s.react()
    nb1 = np.bincount(s.key, weights=(s.flags & 1), minlength=s.ncells)
    assert np.array_equal(nb0 - nb1, (nb0 > 0).astype(float))


def test_bulk_reaction_rate_and_uniform_choice(orc):
    k, tau = 0.05, 0.5
    cfg = synth.base_config(L=(4, 4, 4), bulk_rate=k, tau=tau)
    s = _cells(orc, cfg, 0.4, 5)
    f0 = s.flags.copy()
    nb = np.bincount(s.key, weights=(f0 & 1), minlength=s.ncells)
    expect = np.sum(1.0 - np.exp(-k * nb * tau))
    hits = []
    picks = np.zeros(s.n)
    for step in range(3000):
        s.flags = f0.copy()
        s.step_index = step
        s.react()
        changed = np.nonzero(s.flags != f0)[0]
        hits.append(len(changed))
        picks[changed] += 1
    hits = np.asarray(hits, float)
    se = hits.std() / math.sqrt(len(hits))
    assert abs(hits.mean() - expect) < 4 * se + 1e-9
    # only B particles ever change, and within a cell each B is equally likely
    assert not np.any(picks[(f0 & 1) == 0])
    from scipy import stats
    pvals = []
    for c in range(s.ncells):
        sl = np.arange(s.start[c], s.start[c] + s.count[c])
        bs = sl[(f0[sl] & 1) == 1]
        if len(bs) >= 3 and picks[bs].sum() > 40:
            pvals.append(stats.chisquare(picks[bs]).pvalue)
    assert len(pvals) > 10
    assert stats.kstest(pvals, "uniform").pvalue > 1e-3
