"""The C twin of the R-MAT recipe returns exactly the bytes of gen.rmat (numpy)."""
import numpy as np
import pytest

from paper_2201_02789_gb300 import build, gen


@pytest.fixture(scope="module", autouse=True)
def native_lib():
    build.build_gen()
    assert gen.native_available()


@pytest.mark.parametrize("scale,n,ef,seed,weights", [
    (8, None, 16, 2, (1, 255)),        # full 2^scale range: only self-loops redrawn
    (10, 600, 8, 11, (1, 255)),        # n < 2^scale: out-of-range endpoints redrawn over many attempts
    (11, 1025, 20, 4000007, None),     # just above a power of two (most redraws), no weights
    (5, 17, 32, 3, (7, 9)),            # tiny, heavy duplication
])
def test_native_matches_numpy(scale, n, ef, seed, weights):
    a = gen.rmat(scale, ef, seed=seed, n=n, weights=weights, native=False)
    b = gen.rmat(scale, ef, seed=seed, n=n, weights=weights, native=True)
    assert a.n == b.n and a.m == b.m
    np.testing.assert_array_equal(a.row_ptr, b.row_ptr)
    np.testing.assert_array_equal(a.col, b.col)
    if weights is None:
        assert b.w is None
    else:
        np.testing.assert_array_equal(a.w, b.w)


def test_batch_instances_match():
    specs = [s for s in gen.batch_specs(64, seed=4, log2_lo=6.0, log2_hi=12.0)][:24]
    nat = gen.batch_graphs(specs)
    for s, g in zip(specs, nat):
        ref = gen.batch_instance(s, native=False)
        np.testing.assert_array_equal(ref.row_ptr, g.row_ptr)
        np.testing.assert_array_equal(ref.col, g.col)
        np.testing.assert_array_equal(ref.w, g.w)
