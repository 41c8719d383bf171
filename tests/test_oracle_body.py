"""Pins of the oracle's rigid bead body (the Janus particle of §1.5, whose
bead network §1.4 holds rigid): free rotation against closed forms and an
independent ODE integration, force and torque against derivatives of the
energy, conservation of momentum, angular momentum and energy over an
interval, the near-list reach, and catalysis on the catalytic hemisphere."""
import math

import numpy as np
import pytest

from paper_1608_04904_gb300 import synth


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _axis_quat(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * axis])


def _rand_quat(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


def test_quaternion_matrix_is_a_rotation(orc):
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(20):
        q = _rand_quat(rng)
        R = orc.quat_matrix(q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        # rotation by angle a about n turns n to itself and a perpendicular u by a
        n = q[1:] / np.linalg.norm(q[1:])
        a = 2 * math.atan2(np.linalg.norm(q[1:]), q[0])
        assert np.allclose(R @ n, n, atol=1e-14)
        u = np.cross(n, [1.0, 0.0, 0.0])
        u /= np.linalg.norm(u)
        assert abs(float(u @ (R @ u)) - math.cos(a)) < 1e-13
    # composition: matrix of a product is the product of the matrices
    a, b = _rand_quat(rng), _rand_quat(rng)
    assert np.allclose(orc.quat_matrix(_qmul(a, b)), orc.quat_matrix(a) @ orc.quat_matrix(b), atol=1e-14)
    # matrix_quaternion of the input generator inverts it
    q = _rand_quat(rng)
    q2 = synth.matrix_quaternion(orc.quat_matrix(q))
    assert np.allclose(q2 * np.sign(q2[0]), q * np.sign(q[0]), atol=1e-14)


def test_rotation_about_a_principal_axis_is_uniform(orc):
    """l along principal axis k: the body turns about e_k at omega = l_k / I_k,
    l stays fixed (closed form; the Cayley angle is exact to O((omega dt)^3))."""
    I = np.array([2.0, 3.0, 5.0])
    dt, n = 0.01, 400
    for k in range(3):
        l0 = np.zeros(3)
        l0[k] = 7.0
        q, l = orc.body_rotate(I, dt, [1, 0, 0, 0], l0, steps=n)
        w = l0[k] / I[k]
        e = np.zeros(3)
        e[k] = 1.0
        exact = _axis_quat(e, w * n * dt)
        tol = n * (w * dt) ** 3 / 12 + 1e-12
        assert np.allclose(q, exact, atol=tol)
        assert np.array_equal(l, l0)


def test_free_rotation_conserves_space_angular_momentum(orc):
    """Every sub-rotation turns q by +phi and l by -phi about the same axis, so
    L = R(q) l is conserved to rounding; |q| = 1; the kinetic energy of the
    symplectic splitting only oscillates at O(dt^2)."""
    rng = np.random.Generator(np.random.PCG64(11))
    I = np.array([1.0, 2.0, 3.5])
    q = _rand_quat(rng)
    l = rng.standard_normal(3) * 3.0
    L0 = orc.quat_matrix(q) @ l
    E0 = 0.5 * (l * l / I).sum()
    dt = 0.02
    for i in range(20):
        q, l = orc.body_rotate(I, dt, q, l, steps=50)
        assert np.allclose(orc.quat_matrix(q) @ l, L0, rtol=0, atol=1e-12 * np.linalg.norm(L0) * (i + 1))
        assert abs(np.linalg.norm(q) - 1) < 1e-14
        assert abs(0.5 * (l * l / I).sum() - E0) < 0.05 * E0 * (dt * np.linalg.norm(l) / I.min()) ** 2 + 1e-12


def test_symmetric_top_precession_second_order(orc):
    """I1 = I2: in the body frame l3 is constant and (l1, l2) turns at
    Omega = l3 (1/I3 - 1/I1) (Euler's equations); the splitting converges to
    it at second order (its turns about e_1, e_2 move l3 at O(dt^2) only)."""
    I = np.array([2.0, 2.0, 5.0])
    a, c = 1.5, 4.0
    T = 3.0
    Om = c * (1 / I[2] - 1 / I[0])
    exact = np.array([a * math.cos(Om * T), -a * math.sin(Om * T), c])
    errs = []
    for dt in (0.02, 0.01):
        _, l = orc.body_rotate(I, dt, [1, 0, 0, 0], [a, 0.0, c], steps=int(round(T / dt)))
        assert abs(l[2] - c) < 1e-4
        errs.append(np.linalg.norm(l - exact))
    assert errs[1] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_asymmetric_top_matches_ode_integration(orc):
    """Against a tight-tolerance Runge-Kutta integration of Euler's equations
    dl/dt = l x (l / I) and of dq/dt = q (0, l / I) / 2: second-order error."""
    integrate = pytest.importorskip("scipy.integrate")
    I = np.array([1.0, 2.0, 3.5])
    rng = np.random.Generator(np.random.PCG64(5))
    q0 = _rand_quat(rng)
    l0 = np.array([0.7, 1.9, -1.2])
    T = 2.0

    def rhs(t, y):
        q, l = y[:4], y[4:]
        w = l / I
        return np.concatenate([0.5 * _qmul(q, np.concatenate([[0.0], w])), np.cross(l, w)])

    sol = integrate.solve_ivp(rhs, (0, T), np.concatenate([q0, l0]), method="DOP853", rtol=1e-12, atol=1e-13)
    qe, le = sol.y[:4, -1], sol.y[4:, -1]
    qe /= np.linalg.norm(qe)
    errs = []
    for dt in (0.01, 0.005):
        q, l = orc.body_rotate(I, dt, q0, l0, steps=int(round(T / dt)))
        errs.append(np.linalg.norm(q - qe) + np.linalg.norm(l - le))
    assert errs[1] < 1e-4
    assert 3.0 < errs[0] / errs[1] < 5.0


def _shell_solvent(body, n, rng, r_lo, r_hi, L):
    c = np.asarray(body["x"])
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = rng.uniform(r_lo, r_hi, n)
    return np.mod(c + u * r[:, None], L)


def test_body_force_and_torque_are_energy_derivatives(orc):
    """F = -dU/dX and T . e_k = -dU/dtheta_k for a turn of the body about the
    space axis e_k through its centre (central differences)."""
    body = synth.janus_body(60, (8.0, 8.0, 8.0), seed=2, radius=2.5, eps_A=1.0, eps_B=0.3)
    cfg = synth.base_config(L=(16, 16, 16), seed=2)
    rng = np.random.Generator(np.random.PCG64(8))
    # outside every bead's core (no bead closer than 0.92 sigma), inside the cut-off of some
    x = _shell_solvent(body, 300, rng, 2.5 + 0.92, 2.5 + 1.12, 16)
    flags = (rng.uniform(size=300) < 0.5).astype(np.uint8)
    B = orc.Body(body)
    _, F, T, _ = orc.body_forces(cfg, x, flags, B)
    assert np.linalg.norm(F) > 1 and np.linalg.norm(T) > 1
    h = 1e-5
    for k in range(3):
        Bp, Bm = orc.Body(body), orc.Body(body)
        Bp.x[k] += h
        Bm.x[k] -= h
        dU = (orc.body_forces(cfg, x, flags, Bp)[3] - orc.body_forces(cfg, x, flags, Bm)[3]) / (2 * h)
        assert abs(F[k] + dU) < 1e-5 * max(1.0, abs(dU))
        e = np.zeros(3)
        e[k] = 1.0
        Bp, Bm = orc.Body(body), orc.Body(body)
        Bp.q = _qmul(_axis_quat(e, h), B.q)
        Bm.q = _qmul(_axis_quat(e, -h), B.q)
        dU = (orc.body_forces(cfg, x, flags, Bp)[3] - orc.body_forces(cfg, x, flags, Bm)[3]) / (2 * h)
        assert abs(T[k] + dU) < 1e-5 * max(1.0, abs(dU))


def _janus_cluster(seed, n=400, nb=80, radius=3.0):
    """A body at the centre of a 32^3 box with solvent in a shell around it
    (nothing near the box faces, so no image ever interacts)."""
    cfg = synth.base_config(L=(32, 32, 32), n_md=50, tau=0.5, kT=1.0, seed=seed, skin=1.0)
    body = synth.janus_body(nb, (16.0, 16.0, 16.0), seed=seed, radius=radius, eps_A=1.0, eps_B=0.5)
    body["l"] = body["l"] * 20.0          # a fast spin makes torque errors visible
    rng = np.random.Generator(np.random.PCG64(seed))
    x = _shell_solvent(body, n, rng, radius + 0.92, radius + 2.5, 32)
    v = rng.standard_normal((n, 3))
    flags = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    return cfg, body, x, v, flags


def _totals(orc, s):
    B = s.body
    M, I = B.inertia()
    P = s.v.sum(0) + M * B.v
    J = np.cross(s.x, s.v).sum(0) + M * np.cross(B.x, B.v) + B.matrix() @ B.l
    E = s.kinetic_energy() + s.potential_energy()
    return P, J, E


def test_interval_conserves_momentum_angular_momentum_energy(orc):
    """All pair forces are central, so an interval of velocity Verlet +
    rigid-body splitting conserves total momentum and total angular momentum
    (solvent orbital + body orbital + spin) up to the fixed-point rounding of
    the force sums, and energy to O(dt^2)."""
    cfg, body, x, v, flags = _janus_cluster(4)
    s = orc.OracleSystem(cfg, x, v, flags=flags, body=body)
    P0, J0, E0 = _totals(orc, s)
    for _ in range(4):
        s.interval(all_substep=True)
        P, J, E = _totals(orc, s)
        assert np.allclose(P, P0, rtol=0, atol=1e-8)
        assert np.allclose(J, J0, rtol=0, atol=1e-7 * max(1.0, np.linalg.norm(J0)))
        assert abs(E - E0) < 2e-3 * abs(E0)
    assert np.linalg.norm(s.body.v) > 0 and not np.allclose(s.body.q, body["q"])


def test_near_list_reach_covers_every_interaction(orc):
    """Free flight for the particles outside the reach gives the same interval
    as sub-stepping every particle (equal in exact arithmetic): the bounding
    sphere max|b| + r_c plus |v| tau + skin misses no interaction."""
    cfg, body, x, v, flags = _janus_cluster(6, n=600)
    x = np.concatenate([x, np.random.Generator(np.random.PCG64(1)).uniform(0, 32, (300, 3))])
    v = np.concatenate([v, np.random.Generator(np.random.PCG64(2)).standard_normal((300, 3))])
    flags = np.concatenate([flags, np.zeros(300, np.uint8)])
    a = orc.OracleSystem(cfg, x, v, flags=flags, body=body)
    b = orc.OracleSystem(cfg, x, v, flags=flags, body=body)
    a.interval()
    b.interval(all_substep=True)
    assert 0 < a.near.sum() < len(x)
    assert np.allclose(a.x, b.x, atol=1e-10) and np.allclose(a.v, b.v, atol=1e-10)
    assert np.array_equal(a.flags, b.flags)
    for k in ("x", "v", "q", "l"):
        assert np.allclose(getattr(a.body, k), getattr(b.body, k), atol=1e-10)
    reach = orc.body_reach(body["b"], body["sigma"])
    assert abs(reach - (np.sqrt((body["b"] ** 2).sum(1)).max() + 2 ** (1 / 6) * body["sigma"])) < 1e-14


def test_catalysis_on_the_catalytic_hemisphere_only(orc):
    """An A particle leaving a catalytic bead's range becomes B; one leaving
    a bead of the other hemisphere stays A (§1.5 with p = 1)."""
    cfg = synth.base_config(L=(24, 24, 24), n_md=50, tau=0.5, kT=1.0, seed=9, cat_prob=1.0)
    body = synth.janus_body(120, (12.0, 12.0, 12.0), seed=9, radius=4.0, thermal=False)
    R = orc.quat_matrix(body["q"])
    rb = body["b"] @ R.T
    cat = body["catalytic"]
    jc = int(np.argmax(np.where(cat == 1, rb[:, 2], -np.inf)))     # catalytic pole bead
    jn = int(np.argmin(np.where(cat == 0, rb[:, 2], np.inf)))      # inert pole bead
    xs, vs = [], []
    for j in (jc, jn):
        u = rb[j] / np.linalg.norm(rb[j])
        xs.append(np.asarray(body["x"]) + rb[j] + 1.0 * u)        # inside r_c = 1.12
        vs.append(2.0 * u)                                          # leaves within ~0.06
    s = orc.OracleSystem(cfg, np.array(xs), np.array(vs), body=body)
    s.interval()
    assert s.near.all()
    assert s.flags[0] == 1          # converted to B, tag cleared
    assert s.flags[1] == 0          # still A, never tagged
