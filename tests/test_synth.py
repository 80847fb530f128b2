"""The seeded generators: reproducible, right shape, right density, and
consistent with the oracle's decoder on the bit layout."""
import numpy as np

import oracle
import synth


def test_reproducible_and_shaped():
    a = synth.many_criteria(5, 8, 100_003)[0]
    b = synth.many_criteria(5, 8, 100_003)[0]
    assert len(a) == 8
    for x, y in zip(a, b):
        assert x.dtype == np.uint64 and x.size == synth.nwords(100_003)
        assert np.array_equal(x, y)
        # bits past r are zero
        assert int(x[-1]) >> (100_003 % 64) == 0


def test_densities():
    r = 1 << 20
    for p in (1e-3, 0.05, 0.3):
        w = synth.bernoulli(0, 1, r, p)
        d = synth.words_to_bits(w, r).mean()
        assert abs(d - p) < 6 * np.sqrt(p / r) + 1e-4
        if p >= 0.05:  # enough runs in 2^20 rows for a tight check
            w = synth.clustered(0, 2, r, p)
            d = synth.words_to_bits(w, r).mean()
            assert 0.8 * p < d < 1.25 * p


def test_layout_matches_oracle_decoder():
    rng = np.random.default_rng(3)
    r = 5000
    rows = np.unique(rng.integers(0, r, size=300))
    w = synth.rows_to_words(rows, r)
    assert np.array_equal(oracle.decode(oracle.encode(w, r), r), rows)
    assert np.array_equal(np.nonzero(synth.words_to_bits(w, r))[0], rows)
