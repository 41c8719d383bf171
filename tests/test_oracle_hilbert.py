"""Pins of the oracle's Hilbert order of the cells (§1.4 sorts the solvent by
compact Hilbert indices): at order 1 the curve is the reflected Gray code;
at every order it is a bijection onto [0, 8^m) whose consecutive cells are
face neighbours, starting at the origin, and whose aligned sub-cubes fill
contiguous index ranges; the ranks of a box of any size are a permutation
that follows the curve."""
import numpy as np
import pytest


def _curve(orc, m):
    n = 1 << m
    cells = [(x, y, z) for x in range(n) for y in range(n) for z in range(n)]
    h = np.array([orc.hilbert_index(m, *c) for c in cells])
    order = np.argsort(h)
    return h, np.array(cells)[order]


def test_order_one_is_the_gray_code(orc):
    """The eight corners in index order: bits (x, y, z) of g(i) = i xor (i >> 1)."""
    _, path = _curve(orc, 1)
    gray = [i ^ (i >> 1) for i in range(8)]
    assert [tuple(p) for p in path] == [((g >> 2) & 1, (g >> 1) & 1, g & 1) for g in gray]


@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_curve_is_a_continuous_bijection(orc, m):
    h, path = _curve(orc, m)
    assert np.array_equal(np.sort(h), np.arange(8 ** m))
    steps = np.abs(np.diff(path, axis=0)).sum(1)
    assert np.all(steps == 1)                      # consecutive cells share a face
    assert tuple(path[0]) == (0, 0, 0)


@pytest.mark.parametrize("m", [3, 4])
def test_aligned_subcubes_are_contiguous(orc, m):
    """Every run of 8^k consecutive indices starting at a multiple of 8^k
    covers exactly one aligned cube of side 2^k."""
    _, path = _curve(orc, m)
    for k in range(1, m):
        s = 1 << k
        for start in range(0, 8 ** m, 8 ** k):
            blk = path[start:start + 8 ** k]
            lo = blk.min(0)
            assert np.all(lo % s == 0) and np.all(blk.max(0) - lo == s - 1)


@pytest.mark.parametrize("L", [(12, 10, 6), (5, 7, 6), (16, 16, 16)])
def test_ranks_of_a_box_follow_the_curve(orc, L):
    rank = orc.hilbert_rank(L)
    n = int(np.prod(L))
    assert np.array_equal(np.sort(rank), np.arange(n))
    m = int(np.ceil(np.log2(max(L))))
    c = np.arange(n)
    xyz = np.stack([c % L[0], (c // L[0]) % L[1], c // (L[0] * L[1])], 1)
    h = np.array([orc.hilbert_index(m, *p) for p in xyz])
    assert np.array_equal(np.argsort(rank), np.argsort(h, kind="stable"))
    # locality: cells next in rank are next in space, apart from the curve's
    # excursions outside the box
    path = xyz[np.argsort(rank)]
    steps = np.abs(np.diff(path, axis=0)).sum(1)
    assert np.mean(steps == 1) > 0.8


def _by_id(o):
    k = np.argsort(o.id)
    return o.x[k], o.v[k], o.flags[k]


@pytest.mark.parametrize("setup", ["dimer_bulk_slabs", "channel"])
def test_hilbert_storage_order_changes_no_physics(orc, setup):
    """The storage order of the cells is memory layout only: with the cells
    in Hilbert order the same steps give the same state, bit for bit, once
    matched by particle id; and storage runs by (Hilbert rank of the cell
    key, id).  (Keying a cell's draws by its rank instead of its key would
    change the velocities; the GPU path's parity tests in Hilbert order rest
    on this equality.)"""
    from paper_1608_04904_gb300 import synth
    if setup == "dimer_bulk_slabs":
        cfg, col, bonds = synth.dimer32(precision="fp64", seed=7, L=16)
        cfg = dict(cfg, slabs=[(0.0, 3.0, 1.3), (8.0, 11.0, 0.7)], bulk_rate=0.05)
        x, v, f = synth.solvent(cfg, col, seed=8, frac_b=0.3)
        kw = dict(colloids=synth.colloid_arrays(col), bonds=bonds)
    else:
        cfg = synth.base_config(L=(10, 6, 7), walls=1, rho_wall=10, g=(0.002, 0.0, 0.0), tau=1.0, seed=9,
                                precision="fp64", bulk_rate=0.02)
        x, v, f = synth.solvent(cfg, seed=10, frac_b=0.4)
        kw = {}
    a = orc.OracleSystem(cfg, x, v, f, **kw)
    b = orc.OracleSystem(cfg, x, v, f, cell_order="hilbert", **kw)
    a.step(3)
    b.step(3)
    for p, q in zip(_by_id(a), _by_id(b)):
        assert np.array_equal(p, q)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.V, b.V)
    r = b.rank[b.key]
    assert np.all(np.diff(r) >= 0)
    same = np.diff(r) == 0
    assert np.all(np.diff(b.id.astype(np.int64))[same] > 0)
    assert not np.array_equal(a.key, b.key)   # the orders do differ
