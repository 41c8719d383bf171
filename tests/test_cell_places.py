"""The library's cell places (rmpcd_cell_places, host code, no GPU): linear
order is the identity; Hilbert order equals the oracle's independent
implementation of the compact Hilbert rank (box shapes cubic and not, a
power of two and not, with a wall layer), and consecutive places are face
neighbours wherever the box is a power-of-two cube."""
import numpy as np
import pytest

from paper_1608_04904_gb300 import api, build


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    api.load()


@pytest.mark.parametrize("dims", [(8, 8, 8), (16, 16, 16), (12, 10, 14), (16, 20, 24), (32, 16, 17), (5, 3, 2),
                                  (48, 48, 48), (1, 1, 1)])
def test_hilbert_places_equal_the_oracle(orc, dims):
    got = api.cell_places(dims, "hilbert")
    want = orc.hilbert_rank(dims)
    assert np.array_equal(got, want)
    assert np.array_equal(api.cell_places(dims, "linear"), np.arange(int(np.prod(dims))))


def test_hilbert_places_walk_face_neighbours():
    dims = (16, 16, 16)
    place = api.cell_places(dims, "hilbert")
    key = np.argsort(place)
    x, y, z = key % 16, (key // 16) % 16, key // 256
    steps = np.abs(np.diff(x)) + np.abs(np.diff(y)) + np.abs(np.diff(z))
    assert np.all(steps == 1)


def test_cell_places_rejects_bad_arguments():
    with pytest.raises(api.RmpcdError):
        api.cell_places((0, 4, 4))
    with pytest.raises(KeyError):
        api.cell_places((4, 4, 4), "morton")
