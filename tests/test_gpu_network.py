"""GPU parity of the bead-network Janus particle under iterative RATTLE (the
paper's Janus integrator, §1.4, §1.5): the colour-parallel kernel against the
oracle's sequential sweep over the links listed colour by colour
(orc_interval_network), bit for bit on the FP64 path -- the interval alone,
fused steps with the collision, and a batch of replicas."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1608_04904_gb300 import api, build, network, synth
from parity_util import compare_step

pytestmark = pytest.mark.gpu

TOL, SWEEPS = 1e-12, 10000


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()


def _janus_net(side, seed, nb=120):
    """A Janus network (beads of the rigid construction moving with its
    thermal velocity and spin), its solvent, and links in colour order."""
    cfg, body = synth.batch_janus(side, seed, precision="fp64", nb=nb)
    x, v, fl = synth.solvent(cfg, synth.body_exclusion(body), seed=seed + 50, frac_b=0.1)
    b = np.asarray(body["b"])
    links, d = synth.bead_links(b)
    colors = network.color_links(links, len(b))
    order = network.order_by_color(links, colors)
    links = [links[k] for k in order]
    d = np.asarray(d)[order]
    colors = np.asarray(colors)[order]
    net = orc.Network.from_body(body, links, d)
    return cfg, x, v, fl, net, links, d, colors


def _gpu(reps):
    s = api.System([dict(cfg=r[0], n=len(r[1])) for r in reps], precision="fp64", bucket_cap=0)
    for i, (cfg, x, v, fl, net, links, d, colors) in enumerate(reps):
        s.set_state(i, x, v, fl)
        s.set_network(i, net.xb, net.vb, net.mb, net.epsA, net.epsB, net.cat, net.sigma, links, d, colors,
                      TOL, SWEEPS)
    return s


def _oracle_interval(cfg, x, v, fl, ids, net, step):
    x, v, fl = x.copy(), v.copy(), fl.copy()
    rc, near = orc.interval_network(cfg, x, v, fl, ids, net, step=step, tol=TOL, max_sweeps=SWEEPS)
    assert rc == 0
    return x, v, fl, near


def test_network_interval_bit_exact():
    rep = _janus_net(16, 3)
    cfg, x, v, fl, net, links, d, colors = rep
    assert colors.max() >= 3 and len(links) > 2 * len(net.mb)
    s = _gpu([rep])
    s.set_step(3)
    s.stream_interval()
    st = s.get_state(0)
    xb, vb = s.get_network(0)
    ox, ov, of, near = _oracle_interval(cfg, x, v, fl, np.arange(len(x), dtype=np.uint32), net, 3)
    assert near.sum() > 1000
    assert np.array_equal(st["x"], ox) and np.array_equal(st["v"], ov) and np.array_equal(st["flags"], of)
    assert np.array_equal(xb, net.xb) and np.array_equal(vb, net.vb)
    # the links hold and the network turned
    for (a, b), dl in zip(links, d):
        assert abs(np.linalg.norm(xb[a] - xb[b]) - dl) <= 1e-10 * dl
    assert (of != fl).sum() > 0   # catalysis happened
    s.close()


def test_network_fused_steps_bit_exact():
    rep = _janus_net(16, 5)
    cfg, x, v, fl, net, links, d, colors = rep
    s = _gpu([rep])
    s.set_step(7)
    o = orc.OracleSystem(cfg, x, v, fl, step=7)
    for _ in range(3):
        s.step(1)
        rc, _ = orc.interval_network(cfg, o.x, o.v, o.flags, o.id, net, step=o.step_index, tol=TOL,
                                     max_sweeps=SWEEPS)
        assert rc == 0
        o.shift_and_sort()
        o.collide()
        o.react()
        o.step_index += 1
        compare_step(cfg, s.get_state(0), o, "fp64")
        xb, vb = s.get_network(0)
        assert np.array_equal(xb, net.xb) and np.array_equal(vb, net.vb)
    s.close()


def test_network_batch_equals_oracle_per_replica():
    reps = [_janus_net(side, 11 + i, nb=nb) for i, (side, nb) in enumerate([(16, 100), (20, 160), (24, 220)])]
    s = _gpu(reps)
    s.step(2)
    for i, (cfg, x, v, fl, net, links, d, colors) in enumerate(reps):
        o = orc.OracleSystem(cfg, x, v, fl)
        for _ in range(2):
            rc, _ = orc.interval_network(cfg, o.x, o.v, o.flags, o.id, net, step=o.step_index, tol=TOL,
                                         max_sweeps=SWEEPS)
            assert rc == 0
            o.shift_and_sort()
            o.collide()
            o.react()
            o.step_index += 1
        compare_step(cfg, s.get_state(i), o, "fp64")
        xb, vb = s.get_network(i)
        assert np.array_equal(xb, net.xb) and np.array_equal(vb, net.vb)
    s.close()


def test_network_rejected_where_it_does_not_apply():
    rep = _janus_net(16, 3)
    cfg, x, v, fl, net, links, d, colors = rep
    m = api.System([dict(cfg=cfg, n=len(x))], precision="mixed", bucket_cap=0)
    with pytest.raises(api.RmpcdError) as e:
        m.set_network(0, net.xb, net.vb, net.mb, net.epsA, net.epsB, net.cat, net.sigma, links, d, colors)
    assert e.value.code == "EINVAL"
    m.close()
    s = api.System([dict(cfg=cfg, n=len(x))], precision="fp64", bucket_cap=0)
    bad = np.asarray(colors).copy()
    a0, b0 = links[0]
    k = next(k for k, (a, b) in enumerate(links) if k > 0 and (a in (a0, b0) or b in (a0, b0)))
    bad[k] = bad[0]   # two links at one bead in one colour
    with pytest.raises(api.RmpcdError) as e:
        s.set_network(0, net.xb, net.vb, net.mb, net.epsA, net.epsB, net.cat, net.sigma, links, d, bad)
    assert e.value.code == "EINVAL"
    s.close()
