"""The link colouring of a bead network (paper_1608_04904_gb300.network): a
valid edge colouring, and a colour-by-colour parallel sweep of the iterative
RATTLE position stage -- modelled here with every link of a colour updated
at once from the same positions, as one thread per link would -- equals the
oracle's sequential sweep over the links listed colour by colour, bit for
bit."""
import numpy as np

from paper_1608_04904_gb300 import network, synth


def _shell(nb=80, factor=1.35):
    x = synth.fibonacci_sphere(nb, 4.0)
    links, d = synth.bead_links(x, factor)
    return x, links, d


def test_coloring_is_valid_and_small():
    for factor in (1.35, 2.0):
        x, links, d = _shell(factor=factor)
        colors = network.color_links(links, len(x))
        deg = np.bincount(np.array(links).ravel(), minlength=len(x))
        assert colors.max() + 1 <= 2 * deg.max() - 1
        for c in range(colors.max() + 1):
            beads = np.array([links[k] for k in np.nonzero(colors == c)[0]]).ravel()
            assert len(beads) == len(np.unique(beads))     # no bead twice in a colour


def _parallel_pos_sweeps(links, d, m, xold, x, v, dt, tol, colors, max_sweeps=10000):
    """Model of a colour-parallel kernel: per colour, all links at once."""
    la = np.array([a for a, _ in links])
    lb = np.array([b for _, b in links])
    x, v = x.copy(), v.copy()
    for sweep in range(1, max_sweeps + 1):
        moved = False
        for c in range(colors.max() + 1):
            k = np.nonzero(colors == c)[0]
            a, b = la[k], lb[k]
            s = x[a] - x[b]
            ro = xold[a] - xold[b]
            d2 = d[k] * d[k]
            diff = d2 - (s[:, 0] * s[:, 0] + s[:, 1] * s[:, 1] + s[:, 2] * s[:, 2])
            act = ~(np.abs(diff) <= 2.0 * tol * d2)
            if not act.any():
                continue
            moved = True
            a, b, s, ro, diff = a[act], b[act], s[act], ro[act], diff[act]
            wa, wb, idt = 1.0 / m[a], 1.0 / m[b], 1.0 / dt   # inverse-mass form
            inv = wa + wb
            sro = s[:, 0] * ro[:, 0] + s[:, 1] * ro[:, 1] + s[:, 2] * ro[:, 2]
            g = diff / (2.0 * sro * inv)
            ca = (g * wa)[:, None] * ro
            cb = (g * wb)[:, None] * ro
            x[a] = x[a] + ca
            x[b] = x[b] - cb
            v[a] = v[a] + ca * idt
            v[b] = v[b] - cb * idt
        if not moved:
            return x, v, sweep
    return x, v, -1


def test_parallel_colour_sweep_equals_sequential_colour_order(orc):
    x0, links, d = _shell()
    rng = np.random.default_rng(9)
    m = np.full(len(x0), 1.7)
    v = rng.normal(0.0, 0.5, x0.shape) + np.cross([0.2, -0.1, 0.4], x0)
    dt, tol = 0.02, 1e-13
    x = x0 + dt * v
    colors = network.color_links(links, len(x0))
    order = network.order_by_color(links, colors)
    links_c = [links[k] for k in order]
    xs, vs, ns = orc.rattle_pos_iter(links_c, d[order], m, x0, x, v, dt, tol=tol)
    xp, vp, npar = _parallel_pos_sweeps(links_c, d[order], m, x0, x, v, dt, tol, colors[order])
    assert ns > 0 and npar == ns
    assert np.array_equal(xp, xs) and np.array_equal(vp, vs)
    # and the colour order reaches the constraint surface like any order
    r = xs[[a for a, _ in links]] - xs[[b for _, b in links]]
    assert np.all(np.abs((r * r).sum(1) - d * d) <= 2 * tol * d * d * 1.0001)


def test_coloring_rejects_bad_links():
    import pytest
    with pytest.raises(ValueError):
        network.color_links([(0, 0)], 3)
    with pytest.raises(ValueError):
        network.color_links([(0, 3)], 3)
    # a triangle needs three colours, a path two
    assert sorted(network.color_links([(0, 1), (1, 2), (0, 2)], 3).tolist()) == [0, 1, 2]
    assert network.color_links([(0, 1), (1, 2), (2, 3)], 4).tolist() == [0, 1, 0]
