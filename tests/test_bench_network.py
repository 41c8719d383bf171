"""The bead-network workload of bench.py on CPU: the replicas are those of
the Janus batch with each Janus particle as a rigid bead network (at least
3 nb - 6 links, a valid edge colouring), and the oracle leg runs its
intervals with every RATTLE stage converged and the links held."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1608_04904_gb300 import network  # noqa: E402


def test_network_workload_is_the_batch_with_rigid_networks():
    reps, desc = bench.workload("network64", "fp64", n_replicas=6)
    base, _ = bench.workload("batch256", "fp64", n_replicas=6)
    assert len(reps) == 6 and "bead network" in desc
    for (cfg, col, bonds, body), (cfg0, _, _, body0) in zip(reps, base):
        assert cfg["L"] == cfg0["L"] and cfg["seed"] == cfg0["seed"] and cfg["precision"] == "fp64"
        net = body["network"]
        nb = len(net["xb"])
        assert nb == len(body0["b"])
        assert len(net["links"]) >= 3 * nb - 6                 # rigid
        colors = network.color_links(net["links"], nb)
        for c in range(colors.max() + 1):
            beads = np.array([net["links"][k] for k in np.nonzero(colors == c)[0]]).ravel()
            assert len(beads) == len(np.unique(beads))
        # links of the construction: their lengths are the bead distances
        a = np.array([p for p, _ in net["links"]])
        b = np.array([q for _, q in net["links"]])
        assert np.allclose(np.linalg.norm(net["xb"][a] - net["xb"][b], axis=1), net["d"], rtol=0, atol=1e-12)
        # centred on the body and moving with it
        assert np.allclose(net["xb"].mean(0), body["x"], atol=1e-9)
        assert np.allclose(net["vb"], body["v"])


def test_network_oracle_leg_runs_converged_intervals(orc):
    reps, _ = bench.workload("network64", "fp64", n_replicas=8)
    r = min(range(len(reps)), key=lambda i: np.prod(reps[i][0]["L"]))   # the smallest box
    rep = reps[r]
    st = bench.initial_state(rep)
    o = bench.oracle_system(orc, rep, st)
    o.step(2)   # raises when a RATTLE stage does not converge
    net = o.net
    r2 = ((net.xb[net.la] - net.xb[net.lb]) ** 2).sum(1)
    assert np.all(np.abs(r2 - net.d ** 2) <= 2.0 * 1e-12 * net.d ** 2 * 1.0001)
