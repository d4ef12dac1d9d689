"""The vectorised digest helper used by the full-size GPU tests equals the
Horner definition the digest sink is documented to compute."""
import numpy as np

from gpu_util import digest_rows, digest_rows_pow


def test_power_form_equals_horner():
    rng = np.random.default_rng(7)
    for n in (0, 1, 2, 3, 31, 1000):
        outs = rng.integers(0, 2**32, size=(5, n), dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(digest_rows_pow(outs), digest_rows(outs)), n
    # extreme words: every term wraps
    outs = np.full((2, 257), 0xFFFFFFFF, dtype=np.uint32)
    assert np.array_equal(digest_rows_pow(outs), digest_rows(outs))
