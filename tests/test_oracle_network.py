"""Pins of the oracle's iterative RATTLE for a linked bead network (§1.4 names
RATTLE in its iterative form as the paper's Janus integrator; Andersen 1983):
one link against the closed-form root of its constraint, a Janus shell whose
links all hold with linear and angular momentum conserved, and free rotation
of a rigid cluster converging at second order to the oracle's rigid-body
integrator (an independent method)."""
import numpy as np

from paper_1608_04904_gb300 import synth


def test_single_link_reaches_the_closed_form_root(orc):
    """One link: the beads move along the old bond by g / m so that the new
    bond has length d; g is the root of smaller magnitude of
    |r_new + g r_old (1/m_a + 1/m_b)|^2 = d^2, and the velocities change by
    the same displacement over dt."""
    rng = np.random.default_rng(1)
    ma, mb, d, dt = 3.0, 5.0, 1.7, 0.05
    xold = np.array([[0.2, -0.1, 0.4], [0.2 + d * 0.6, -0.1 + d * 0.8, 0.4]])
    v = rng.normal(size=(2, 3))
    x = xold + dt * v
    xi, vi, n = orc.rattle_pos_iter([(0, 1)], [d], [ma, mb], xold, x, v, dt, tol=1e-15)
    assert n > 0
    ro, rn, w = xold[0] - xold[1], x[0] - x[1], 1.0 / ma + 1.0 / mb
    roots = np.roots([w * w * (ro @ ro), 2.0 * w * (rn @ ro), rn @ rn - d * d]).real
    g = roots[np.argmin(np.abs(roots))]
    assert np.allclose(xi[0], x[0] + g * ro / ma, rtol=0, atol=1e-12)
    assert np.allclose(xi[1], x[1] - g * ro / mb, rtol=0, atol=1e-12)
    assert np.allclose(vi[0], v[0] + g * ro / (ma * dt), rtol=0, atol=1e-10)
    assert np.allclose(vi[1], v[1] - g * ro / (mb * dt), rtol=0, atol=1e-10)
    assert abs(np.linalg.norm(xi[0] - xi[1]) - d) < 1e-13
    # velocity stage: the relative velocity along the bond goes, the centre
    # of mass velocity stays
    vv, nv = orc.rattle_vel_iter([(0, 1)], [d], [ma, mb], xi, vi, tol=1e-15)
    assert nv > 0
    assert abs((vv[0] - vv[1]) @ (xi[0] - xi[1])) < 1e-13
    assert np.allclose(ma * vv[0] + mb * vv[1], ma * vi[0] + mb * vi[1], rtol=0, atol=1e-13)


def _shell(nb=80, radius=4.0):
    x = synth.fibonacci_sphere(nb, radius)
    links, d = synth.bead_links(x)
    return x, links, d


def test_janus_shell_links_hold_and_momenta_are_conserved(orc):
    """A Janus shell (80 beads on a sphere of radius 4, each linked to its
    neighbours) with thermal and rotational velocities and fixed external
    forces: after one step every link holds within the tolerance, the
    momentum changed by exactly dt times the total force, and without forces
    the angular momentum about the origin is unchanged (constraint impulses
    act along bond vectors)."""
    x, links, d = _shell()
    assert len(links) >= 2 * len(x)          # every bead joined to several neighbours
    rng = np.random.default_rng(5)
    m = np.full(len(x), 2.0)
    v = rng.normal(0.0, 0.3, x.shape) + np.cross([0.1, -0.2, 0.3], x)
    F = rng.normal(0.0, 1.0, x.shape)
    dt, tol = 0.02, 1e-13
    # start on the constraint surface: one pass of both stages at rest
    x1, v1, n = orc.network_steps(links, d, m, x, v, dt, 1, F=F, tol=tol)
    assert n > 0
    a = np.array([i for i, _ in links])
    b = np.array([j for _, j in links])
    r = x1[a] - x1[b]
    assert np.all(np.abs((r * r).sum(1) - d * d) <= 2 * tol * d * d * 1.0001)
    assert np.all(np.abs(((v1[a] - v1[b]) * r).sum(1)) <= tol * d * 1.0001)
    p0, p1 = (m[:, None] * v).sum(0), (m[:, None] * v1).sum(0)
    assert np.allclose(p1 - p0, dt * F.sum(0), rtol=0, atol=1e-11)
    x2, v2, n = orc.network_steps(links, d, m, x1, v1, dt, 5, tol=tol)
    assert n > 0
    L1 = (m[:, None] * np.cross(x1, v1)).sum(0)
    L2 = (m[:, None] * np.cross(x2, v2)).sum(0)
    assert np.allclose(L2, L1, rtol=0, atol=1e-9)


def _rigid_reference(x0, w, T, dt_ref, orc):
    """Torque-free rigid motion of equal unit masses at x0 spinning with w,
    by the oracle's rigid-body integrator (principal frame, quaternion)."""
    com = x0.mean(0)
    r = x0 - com
    I = np.eye(3) * (r * r).sum() - r.T @ r
    Ip, E = np.linalg.eigh(I)
    if np.linalg.det(E) < 0:
        E[:, 2] = -E[:, 2]
    bb = r @ E                                 # body-frame positions
    q = synth.matrix_quaternion(E)
    l = Ip * (E.T @ w)                         # body-frame angular momentum
    q, l = orc.body_rotate(Ip, dt_ref, q, l, steps=int(round(T / dt_ref)))
    return com + bb @ orc.quat_matrix(q).T


def test_free_rotation_converges_to_the_rigid_body_at_second_order(orc):
    """Twelve beads joined by all 66 links form a rigid cluster.  Spun up and
    left alone, its iterative-RATTLE motion approaches the rigid-body
    integrator's (run with a much smaller step) with an error that drops by
    four when the step halves, and its kinetic energy stays within O(dt^2)."""
    x0 = synth.fibonacci_sphere(12, 1.5) + np.array([0.3, -0.2, 0.1])
    links = [(i, j) for i in range(12) for j in range(i + 1, 12)]
    d = np.array([np.linalg.norm(x0[i] - x0[j]) for i, j in links])
    m = np.ones(12)
    w = np.array([0.3, -0.7, 1.1])
    v0 = np.cross(w, x0 - x0.mean(0))
    T = 1.0
    ref = _rigid_reference(x0, w, T, 2e-4, orc)
    err, ke = [], []
    for dt in (0.02, 0.01):
        x, v, n = orc.network_steps(links, d, m, x0, v0, dt, int(round(T / dt)), tol=1e-14)
        assert n > 0
        err.append(np.abs(x - ref).max())
        ke.append(0.5 * (m[:, None] * v * v).sum())
    ke0 = 0.5 * (m[:, None] * v0 * v0).sum()
    assert err[1] < 2e-3
    assert 3.0 < err[0] / err[1] < 5.5, err
    assert abs(ke[1] - ke0) < 1e-3 * ke0


def _janus_case(orc, n_md=25, L=16, factor=2.0, seed=4):
    """A spinning 60-bead Janus particle in a 16^3 solvent, as a rigid body and
    as the same beads linked to their neighbours (a rigid shell)."""
    cfg = synth.base_config(L=(L, L, L), alpha=np.radians(130.0), tau=0.5, n_md=n_md, kT=1.0, seed=seed)
    body = synth.janus_body(60, (L / 2 + 0.3, L / 2 - 0.2, L / 2 + 0.1), seed=seed)
    body["l"] = body["l"] * 20.0
    x, v, fl = synth.solvent(cfg, synth.body_exclusion(body), seed=seed + 1, frac_b=0.2)
    xb0 = body["x"] + body["b"] @ orc.quat_matrix(body["q"]).T
    links, d = synth.bead_links(xb0, factor)
    return cfg, body, links, d, x, v, fl


def test_network_interval_conserves_momentum_energy_and_links(orc):
    """One interval of solvent and bead network: total momentum to rounding
    (the reactions are exact fixed-point sums), energy within 1e-4 relative
    (velocity Verlet at dt 0.02), every link held in length and without
    relative velocity along it, no skin violation."""
    cfg, body, links, d, x, v, fl = _janus_case(orc)
    net = orc.Network.from_body(body, links, d)
    ids = np.arange(len(x), dtype=np.uint32)
    p0 = v.sum(0) + net.momentum()
    e0 = 0.5 * (v ** 2).sum() + net.kinetic_energy() + orc.network_energy(cfg, x, fl, net)
    st, near = orc.interval_network(cfg, x, v, fl, ids, net)
    assert st == 0 and near.sum() > 1000
    p1 = v.sum(0) + net.momentum()
    e1 = 0.5 * (v ** 2).sum() + net.kinetic_energy() + orc.network_energy(cfg, x, fl, net)
    assert np.allclose(p1, p0, rtol=0, atol=1e-10)
    assert abs(e1 - e0) < 1e-4 * e0
    r = net.xb[net.la] - net.xb[net.lb]
    assert np.abs(np.sqrt((r * r).sum(1)) - net.d).max() < 1e-10
    # the velocity stage: no relative velocity along any link
    w = net.vb[net.la] - net.vb[net.lb]
    assert np.abs((w * r).sum(1)).max() < 1e-10 * net.d.max()


def test_network_interval_free_flight_equals_substepping(orc):
    """Particles beyond the bounding sphere fly freely; sub-stepping every
    particle instead gives the same beads and near particles bit for bit and
    the far particles within rounding."""
    cfg, body, links, d, x, v, fl = _janus_case(orc)
    ids = np.arange(len(x), dtype=np.uint32)
    out = []
    for all_sub in (False, True):
        net = orc.Network.from_body(body, links, d)
        xs, vs, fs = x.copy(), v.copy(), fl.copy()
        st, near = orc.interval_network(cfg, xs, vs, fs, ids, net, all_substep=all_sub)
        assert st == 0
        out.append((xs, vs, fs, net, near))
    (xa, va, fa, na, near), (xb, vb, fb, nb_, _) = out
    assert np.array_equal(na.xb, nb_.xb) and np.array_equal(na.vb, nb_.vb)
    assert np.array_equal(xa[near], xb[near]) and np.array_equal(va[near], vb[near])
    assert np.array_equal(fa, fb)
    assert np.allclose(xa[~near], xb[~near], rtol=0, atol=1e-12)
    assert np.allclose(va[~near], vb[~near], rtol=0, atol=1e-14)


def test_network_interval_converges_to_the_rigid_body_interval(orc):
    """The linked shell moves as a rigid body, so its interval and the
    rigid-body interval approximate the same motion with two different
    second-order integrators: their solvent states and centres of mass
    differ by O(dt^2) -- a fourth when the sub-step halves -- and the
    catalytic flags agree."""
    diffs = []
    for n_md in (25, 50):
        cfg, body, links, d, x, v, fl = _janus_case(orc, n_md=n_md)
        net = orc.Network.from_body(body, links, d)
        ids = np.arange(len(x), dtype=np.uint32)
        xn, vn, fn = x.copy(), v.copy(), fl.copy()
        st, _ = orc.interval_network(cfg, xn, vn, fn, ids, net, tol=1e-13)
        assert st == 0
        s = orc.OracleSystem(cfg, x.copy(), v.copy(), fl.copy(), body=body)
        s.interval()
        L = cfg["L"][0]
        dx = np.abs(xn - s.x)
        dx = np.minimum(dx, L - dx)
        diffs.append((dx.max(), np.abs(vn - s.v).max(), np.abs(net.com() - s.body.x).max()))
        assert np.array_equal(fn, s.flags)
    for k in range(3):
        assert 3.5 < diffs[0][k] / diffs[1][k] < 4.5, diffs
    assert diffs[1][0] < 1e-6 and diffs[1][1] < 1e-5
