"""The test-side digest of cb_opts.digests (tests/parity.py) on small hand
cases: it must see every part of a product (row lengths, positions, columns,
values; the pattern only for fp64) so that a digest match means something."""
import math

import numpy as np

from parity import _sm64, digest, digest_words, exact_sum


def _case():
    rp = np.array([0, 2, 2, 5], np.int64)
    col = np.array([1, 7, 0, 3, 9], np.int32)
    val = np.array([5, 6, 7, 8, 9], np.uint32)
    return rp, col, val


def test_splitmix64_reference_values():
    # published outputs of splitmix64 seeded with 0 (the state advanced by the
    # golden gamma before each output): 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4
    g = 0x9E3779B97F4A7C15
    assert int(_sm64(np.array([0], np.uint64))[0]) == 0xE220A8397B1DCDAF
    assert int(_sm64(np.array([g], np.uint64))[0]) == 0x6E789E6AA1B965F4


def test_digest_sees_every_part():
    rp, col, val = _case()
    d0, v = digest("min_plus_u32", rp, col, val)
    assert v is None
    variants = []
    c2 = col.copy(); c2[3] = 4
    variants.append((rp, c2, val))                                    # a column
    v2 = val.copy(); v2[0] = 50
    variants.append((rp, col, v2))                                    # a value
    variants.append((np.array([0, 2, 3, 5]), col, val))               # row lengths
    variants.append((np.array([0, 0, 2, 5]), col, val))               # rows swapped
    variants.append((rp, col[[1, 0, 2, 3, 4]], val[[1, 0, 2, 3, 4]]))  # order inside a row
    for r, c, x in variants:
        assert digest("min_plus_u32", r, c, x)[0] != d0


def test_fp64_digest_is_the_pattern_plus_a_weighted_checksum():
    rp, col, _ = _case()
    val = np.array([0.5, -1.25, 3.0, 2.0, -0.75])
    d0, v = digest("plus_times_f64", rp, col, val)
    assert digest("plus_times_f64", rp, col, val * 3)[0] == d0
    # V written out term by term
    terms = []
    rows = [0, 0, 2, 2, 2]
    for e, r in enumerate(rows):
        h = int(_sm64(np.array([2 * r + 1], np.uint64))[0])
        w = 1.0 + float(int(_sm64(np.array([h ^ int(col[e])], np.uint64))[0]) >> 11) * 2.0 ** -53
        assert 1.0 <= w < 2.0
        terms.append(val[e] * w)
    assert v == math.fsum(terms)


def test_digest_words_reads_raw_bits():
    words = np.array([-1, np.float64(2.5).view(np.int64)], np.int64)
    assert digest_words(words, 0) == (2 ** 64 - 1, 2.5)


def test_exact_sum_is_correctly_rounded_where_plain_sums_are_not():
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(100_001) * 10.0 ** rng.integers(-8, 8, 100_001),
                        [1e16, -1e16, 3.0]])
    assert exact_sum(x) == math.fsum(x.tolist())
    assert exact_sum(np.array([1e16, 1.0, -1e16])) == 1.0 != np.sum(np.array([1e16, 1.0, -1e16]))
    assert exact_sum(np.zeros(0)) == 0.0
