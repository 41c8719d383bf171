"""The error path of the bounded waits, exercised without any GPU fault.

A sorting pass of the flat layout (the granular calls, and the flattening of
a fused run's state for state transfer and observables) finds each tile's
output base by waiting for its predecessors' published prefixes (decoupled
look-back); that wait is bounded.  The test
hook rmpcd_set_wait_test(stall) makes every predecessor read as not ready --
a flag that nothing sets -- so each wait runs out after a few polls: the
kernel must return, latch RMPCD_ETIMEOUT for the host, write nothing out of
bounds, and leave the CUDA context usable for a fresh system."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1608_04904_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    api.load()


def _system(precision):
    cfg = synth.base_config(L=(16, 16, 16), precision=precision, seed=3)   # 32 tiles of cells
    x, v, fl = synth.solvent(cfg, seed=5)
    s = api.System.single(cfg, len(x), precision=precision, bucket_cap=0)
    s.set_state(0, x, v, fl)
    return cfg, x, v, fl, s


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_lookback_wait_runs_out_and_reports_etimeout(precision):
    cfg, x, v, fl, s = _system(precision)
    s.step(1)
    s.sync()                                   # a normal interval: no error
    s.set_wait_test(max_polls=1000, stall=True)
    s.step(1)
    s.shift_and_sort()                         # flat sorting passes: every tile but the first gives up
    with pytest.raises(api.RmpcdError) as e:
        s.sync()
    assert e.value.code == "ETIMEOUT", str(e.value)
    assert "look-back" in str(e.value)
    s.close()
    # the context is still usable: a fresh system steps and matches the oracle
    cfg, x, v, fl, s = _system(precision)
    s.step(1)
    st = s.get_state(0)
    o = orc.OracleSystem(cfg, x, v, fl)
    o.step(1)
    assert np.array_equal(np.sort(st["id"]), np.arange(len(x)))
    if precision == "fp64":
        assert np.array_equal(st["id"], o.id) and np.array_equal(st["cell"], o.key)
    s.close()


def test_wait_limit_rejects_negative():
    cfg, x, v, fl, s = _system("mixed")
    with pytest.raises(api.RmpcdError) as e:
        s.set_wait_test(max_polls=-1)
    assert e.value.code == "EINVAL"
    s.set_wait_test(max_polls=0, stall=False)    # back to the default: runs normally
    s.step(2)
    s.shift_and_sort()
    s.sync()
    s.close()
