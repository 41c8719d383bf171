"""Pins of the oracle's grid shift, cell keys and counting sort (§1.4): cells
in key order, particles of a cell in id order."""
import numpy as np

from paper_1608_04904_gb300 import synth


def _brute_cell(x, s, L, walls):
    """Find each particle's cell by scanning the cell boundaries s + k <= x < s + k + 1."""
    out = []
    for xi in x:
        c = []
        for d in range(3):
            if d == 2 and walls:
                found = None
                for k in range(-1, L[2] + 1):
                    if s[d] + k <= xi[d] < s[d] + k + 1:
                        found = k + 1
                        break
                if found is None:
                    found = L[2] if xi[d] >= s[d] + L[2] else 0
                c.append(min(max(found, 0), L[2]))
            else:
                found = None
                for k in range(-1, L[d] + 1):
                    if s[d] + k <= xi[d] < s[d] + k + 1:
                        found = k % L[d]
                        break
                c.append(found)
        out.append(c[0] + L[0] * (c[1] + L[1] * c[2]))
    return np.asarray(out, dtype=np.int32)


def test_cell_keys_match_boundary_scan(orc):
    cfg = synth.base_config(L=(5, 4, 3))
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.integers(0, np.asarray(cfg["L"]) << 24, size=(300, 3)).astype(np.float64) * 2.0**-24
    for step in range(5):
        s = orc.grid_shift(77, step)
        assert np.array_equal(orc.cell_keys(cfg, x, s), _brute_cell(x, s, cfg["L"], False))


def test_cell_keys_with_walls(orc):
    cfg = synth.base_config(L=(4, 3, 5), walls=1, rho_wall=10)
    rng = np.random.Generator(np.random.PCG64(4))
    x = rng.uniform(0, 1, size=(300, 3)) * np.asarray(cfg["L"])
    x[:10, 2] = 0.0
    x[10:20, 2] = 5.0
    assert orc.n_cells(cfg) == 4 * 3 * 6
    for step in range(5):
        s = orc.grid_shift(5, step)
        assert np.array_equal(orc.cell_keys(cfg, x, s), _brute_cell(x, s, cfg["L"], True))


def test_counting_sort_orders_by_cell_then_id(orc):
    """The order is lexicographic in (cell key, particle id), whatever order
    the particles come in (ids unique, not necessarily 0..n-1)."""
    rng = np.random.Generator(np.random.PCG64(5))
    for ncells, n in [(1, 50), (7, 0), (64, 1000), (1000, 300)]:
        key = rng.integers(0, ncells, size=n).astype(np.int32)
        ids = rng.permutation(5 * n)[:n].astype(np.uint32)
        perm, count, start = orc.counting_sort(key, ncells, ids)
        assert np.array_equal(perm, np.lexsort((ids, key)))
        assert np.array_equal(count, np.bincount(key, minlength=ncells))
        assert np.array_equal(start, np.concatenate([[0], np.cumsum(count)[:-1]]) if ncells else start)
        assert count.sum() == n
        # without ids the index is the id: a stable sort by key
        perm0, _, _ = orc.counting_sort(key, ncells)
        assert np.array_equal(perm0, np.argsort(key, kind="stable"))


def test_shift_and_sort_reorders_state(orc):
    cfg = synth.base_config(L=(6, 6, 6))
    x, v, fl = synth.solvent(cfg, n=2000, seed=11, frac_b=0.3)
    s = orc.OracleSystem(cfg, x, v, fl)
    s.shift_and_sort()
    key = orc.cell_keys(cfg, x, orc.grid_shift(cfg["seed"], 0))
    order = np.argsort(key, kind="stable")   # ids are 0..n-1 in input order
    assert np.array_equal(s.id, order)
    assert np.array_equal(s.x, x[order])
    assert np.array_equal(s.flags, fl[order])
    assert np.all(np.diff(s.key) >= 0)
