"""Pins for the oracle's sketch generator (Alg. 2, "Generate i.i.d Gaussian matrix").

Philox4x64-10 is pinned against numpy's own Philox bit generator (a library routine
implementing the same published definition); the Box-Muller map is pinned by the
distribution it must produce.
"""
import numpy as np
import pytest
from scipy import stats

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _numpy_philox_block(ctr, key):
    # numpy's Philox advances the counter by one before producing each 4-word block.
    c = [int(x) for x in ctr]
    prev = (c[0] + (c[1] << 64) + (c[2] << 128) + (c[3] << 192) - 1) % (1 << 256)
    words = np.array([(prev >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=words)
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ([1, 0, 0, 0], [0, 0]),
    ([0, 0, 0, 0], [12345, 0]),
    ([7, 0, 0, 0], [0, 0]),
    ([123456789, 0, 0, 0], [2**64 - 1, 2**63]),
    ([2**64 - 1, 5, 0, 0], [0xDEADBEEF, 17]),
    ([0, 1, 2, 3], [4, 5]),
])
def test_philox_matches_numpy(orc, ctr, key):
    got = orc.philox4x64_10(ctr, key)
    want = _numpy_philox_block(ctr, key)
    assert np.array_equal(got, want)


def test_omega_is_standard_normal(orc):
    Om = orc.omega(80, 40000, seed=0)
    x = Om.ravel()
    assert abs(x.mean()) < 5e-3
    assert abs(x.var() - 1.0) < 5e-3
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # cos/sin halves of each Box-Muller pair are uncorrelated and each standard normal
    even, odd = x[0::2], x[1::2]
    assert abs(np.corrcoef(even, odd)[0, 1]) < 5e-3
    assert stats.kstest(even, "norm").pvalue > 1e-3
    assert stats.kstest(odd, "norm").pvalue > 1e-3
    # squared radius of a pair is exponential with mean 2 (chi-square, 2 d.o.f.)
    r2 = even[0::2] ** 2 + odd[0::2] ** 2
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-3


def test_omega_seed_and_prefix(orc):
    a = orc.omega(8, 100, seed=3)
    b = orc.omega(8, 100, seed=3)
    c = orc.omega(8, 100, seed=4)
    assert np.array_equal(a, b)
    assert not np.allclose(a, c)
    # element q depends only on its flat index: a longer draw starts with the same numbers
    long = orc.omega(1, 800, seed=3).ravel()
    assert np.array_equal(long, a.ravel())
