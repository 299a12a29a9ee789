"""Pins of the oracle's counter-based generator (Alg. 1 draws Omega from it).

The oracle's Philox4x64-10 is checked against NumPy's Philox bit generator, an
independent implementation of the same published definition (NumPy advances
the counter by one before producing a block)."""
import numpy as np
import pytest
from scipy import stats

from oracle import philox as P

MASK = (1 << 64) - 1


def _numpy_block(counter, key):
    c = [int(x) & MASK for x in counter]
    # counter - 1 with borrow across the 256-bit counter
    val = c[0] | (c[1] << 64) | (c[2] << 128) | (c[3] << 192)
    val = (val - 1) % (1 << 256)
    prev = np.array([(val >> (64 * i)) & MASK for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(counter=prev, key=np.array(key, dtype=np.uint64))
    return [int(x) for x in bg.random_raw(4)]


@pytest.mark.parametrize("counter,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((7, 3, 2, 1), (12345, 0)),
    ((0, 5, 0, 0), (2**63 + 11, 1)),          # borrow into the second word
    ((2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1), (2**64 - 1, 2**64 - 1)),
    ((123456789, 42, 7, 999), (0xDEADBEEF, 0xFEEDFACE)),
])
def test_philox_matches_numpy(counter, key):
    assert list(P.philox4x64_10(counter, key)) == _numpy_block(counter, key)


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(3)
    cs = rng.integers(0, 2**63, size=(4, 16), dtype=np.uint64)
    out = P.philox4x64_10_array(cs[0], cs[1], cs[2], cs[3], 987654321, 5)
    for t in range(16):
        ref = P.philox4x64_10((cs[0][t], cs[1][t], cs[2][t], cs[3][t]), (987654321, 5))
        assert [int(o[t]) for o in out] == list(ref)


def test_uniform_open_interval():
    u = P.uniform53(np.array([0, 2**64 - 1], dtype=np.uint64))
    assert u[0] > 0.0 and u[1] < 1.0


def test_gaussian_omega_statistics():
    om = P.gaussian_omega(400, 100, seed=11, bond=3, sweep=5, chain=2)
    re, im = om.real.ravel(), om.imag.ravel()
    for x in (re, im):
        assert abs(x.mean()) < 0.02
        assert abs(x.std() - 1.0) < 0.02
        assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(re, im)[0, 1]) < 0.02


def test_gaussian_omega_counter_layout():
    base = P.gaussian_omega(6, 4, seed=1, bond=2, sweep=3, chain=4)
    # element (r, c) uses counter index r*l + c: a wider matrix re-reads the same stream
    flat = P.gaussian_omega(1, 24, seed=1, bond=2, sweep=3, chain=4).ravel()
    assert np.array_equal(base.ravel(), flat)
    for kw in ({"bond": 3}, {"sweep": 4}, {"chain": 5}, {"stream": 1}):
        args = dict(seed=1, bond=2, sweep=3, chain=4)
        args.update(kw)
        assert not np.allclose(P.gaussian_omega(6, 4, **args), base)
    assert not np.allclose(P.gaussian_omega(6, 4, seed=2, bond=2, sweep=3, chain=4), base)
