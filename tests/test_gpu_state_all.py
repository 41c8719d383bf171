"""The batch state calls (rmpcd_set_state_all / rmpcd_get_state_all): every
replica's solvent in one call, concatenated in replica order, must give
exactly what the per-replica calls give -- before any step (storage order =
input order) and after fused steps (flattened, sorted state) -- from host
arrays and from device arrays, on both precisions; and a wrong total is
rejected."""
import numpy as np
import pytest

from paper_1608_04904_gb300 import api, build, synth

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]
KEYS = ("x", "v", "flags", "id", "cell")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()


def _replicas(precision):
    """A plain replica, a Janus replica and a channel with walls, of different sizes."""
    reps = []
    cfg = synth.base_config(L=(12, 10, 14), seed=21, precision=precision)
    x, v, f = synth.solvent(cfg, seed=22, frac_b=0.3)
    reps.append((dict(cfg=cfg, n=len(x)), (x, v, f)))
    cfg, body = synth.batch_janus(16, 23, precision=precision, nb=110)
    x, v, f = synth.solvent(cfg, synth.body_exclusion(body), seed=24, frac_b=0.2)
    reps.append((dict(cfg=cfg, n=len(x), body=body), (x, v, f)))
    cfg = synth.base_config(L=(10, 12, 9), walls=1, rho_wall=10, g=(0.001, 0.0, 0.0), tau=1.0, seed=25,
                            precision=precision)
    x, v, f = synth.solvent(cfg, seed=26)
    reps.append((dict(cfg=cfg, n=len(x)), (x, v, f)))
    return reps


def _cat(states):
    return tuple(np.concatenate([s[k] for s in states]) for k in range(3))


def _system(reps, precision):
    return api.System([r for r, _ in reps], precision, 64)


@pytest.mark.parametrize("precision", PRECS)
def test_set_all_equals_per_replica_before_any_step(precision):
    reps = _replicas(precision)
    a = _system(reps, precision)
    b = _system(reps, precision)
    for i, (_, st) in enumerate(reps):
        a.set_state(i, *st)
    b.set_state_all(*_cat([st for _, st in reps]))
    whole = b.get_state_all()
    off = 0
    for i, (_, st) in enumerate(reps):
        ga, gb = a.get_state(i), b.get_state(i)
        n = len(st[0])
        for k in KEYS:
            assert np.array_equal(ga[k], gb[k]), (i, k)
            assert np.array_equal(whole[k][off:off + n], ga[k]), (i, k)
        assert np.array_equal(ga["id"], np.arange(n, dtype=np.uint32))
        off += n
    a.close()
    b.close()


@pytest.mark.parametrize("precision", PRECS)
def test_all_calls_equal_per_replica_after_fused_steps(precision):
    reps = _replicas(precision)
    a = _system(reps, precision)
    b = _system(reps, precision)
    for i, (_, st) in enumerate(reps):
        a.set_state(i, *st)
    b.set_state_all(*_cat([st for _, st in reps]))
    a.step(3)
    b.step(3)
    per = [a.get_state(i) for i in range(len(reps))]
    whole = b.get_state_all()
    for k in KEYS:
        assert np.array_equal(np.concatenate([p[k] for p in per]), whole[k]), k
    # a second round trip through the batch calls continues the same run
    b.set_state_all(whole["x"], whole["v"], whole["flags"])
    for i in range(len(reps)):
        a.set_state(i, per[i]["x"], per[i]["v"], per[i]["flags"])
    a.step(2)
    b.step(2)
    whole2 = b.get_state_all()
    for k in KEYS:
        assert np.array_equal(np.concatenate([a.get_state(i)[k] for i in range(len(reps))]), whole2[k]), k
    a.close()
    b.close()


@pytest.mark.parametrize("precision", PRECS)
def test_all_calls_with_device_arrays(precision):
    import torch
    reps = _replicas(precision)
    x, v, f = _cat([st for _, st in reps])
    a = _system(reps, precision)
    b = _system(reps, precision)
    a.set_state_all(x, v, f)
    b.set_state_all(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), torch.from_numpy(f).cuda())
    a.step(2)
    b.step(2)
    host = a.get_state_all()
    n = len(x)
    dev = {"x": torch.empty((n, 3), dtype=torch.float64, device="cuda"),
           "v": torch.empty((n, 3), dtype=torch.float64, device="cuda"),
           "flags": torch.empty(n, dtype=torch.uint8, device="cuda"),
           "id": torch.empty(n, dtype=torch.int32, device="cuda"),
           "cell": torch.empty(n, dtype=torch.int32, device="cuda")}
    b.get_state_all(out=dev)
    torch.cuda.synchronize()
    for k in KEYS:
        got = dev[k].cpu().numpy()
        want = host[k].view(np.int32) if k == "id" else host[k]
        assert np.array_equal(got, want), k
    a.close()
    b.close()


def test_wrong_total_rejected():
    reps = _replicas("mixed")
    s = _system(reps, "mixed")
    x, v, f = _cat([st for _, st in reps])
    for bad in (x[:-1], np.concatenate([x, x[:1]])):
        with pytest.raises(api.RmpcdError) as e:
            s._check(s._lib.rmpcd_set_state_all(s._h, bad.ctypes.data_as(api.C.c_void_p),
                                                v.ctypes.data_as(api.C.c_void_p), None, len(bad), 0))
        assert e.value.code == "EINVAL"
    out = np.empty((len(x) + 1, 3))
    with pytest.raises(api.RmpcdError) as e:
        s._check(s._lib.rmpcd_get_state_all(s._h, out.ctypes.data_as(api.C.c_void_p), None, None, None, None,
                                            len(out), 0))
    assert e.value.code == "EINVAL"
    s.close()
