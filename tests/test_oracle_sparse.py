"""Pins of the sparse sign test matrix oracle (Sec. 3.4)."""
import numpy as np
import pytest

from oracle import gaussian as OG
from oracle import sparse as OSP


def test_threshold_values():
    assert OSP.threshold(1.0) == 2 ** 31                    # no zeros: Rademacher
    assert OSP.threshold(3.0) == 715827883                  # floor(2^32 / 6 + 1/2)
    assert OSP.threshold(2.0 ** 20) == 2048                 # 2^32 / 2^21
    with pytest.raises(ValueError):
        OSP.threshold(0.5)


def test_rademacher_case_is_the_sign_of_the_uniform():
    # s = 1: +1 exactly when the word's uniform (w + 1/2) 2^-32 is below 1/2
    rows, cols = 37, 29
    S = OSP.sparse_sign(5, 3, rows, cols, 1.0)
    u = OG.uniform_open01(OSP.philox_words(5, 3, rows * cols)).reshape(rows, cols)
    assert np.all(S != 0)
    assert np.array_equal(S, np.where(u < 0.5, 1.0, -1.0))


def test_words_are_the_gaussian_stream():
    # the Gaussian generator's first normal of block b is Box-Muller of words 0 and 1
    w = OSP.philox_words(11, 7, 8).astype(np.float64)
    u0 = (w[0] + 0.5) * 2.0 ** -32
    u1 = (w[1] + 0.5) * 2.0 ** -32
    z0 = np.sqrt(-2.0 * np.log(u0)) * np.cos(2.0 * np.pi * u1)
    assert abs(OG.gaussian_f64(11, 7, 1, 4)[0, 0] - z0) < 1e-12


@pytest.mark.parametrize("s", [3.0, 16.0, 128.0])
def test_frequencies(s):
    # nonzero fraction ~ 1/s and sign balance within 5 binomial standard deviations
    n = 400_000
    S = OSP.sparse_sign(2, 0, 1, n, s).ravel()
    p = OSP.threshold(s) / 2.0 ** 32
    for v in (1.0, -1.0):
        c = np.count_nonzero(S == v)
        assert abs(c - n * p) <= 5 * np.sqrt(n * p * (1 - p)), (v, c, n * p)
    assert set(np.unique(S)) <= {-1.0, 0.0, 1.0}
