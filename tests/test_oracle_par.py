"""The piecewise restricted oracle (tests/_oracle_par.py) equals the oracle
run on the whole read set: counts added over pieces with min_count applied to
the sums, filter words OR-ed, windows added."""
import numpy as np

import synth
from tests import _oracle_par


def test_pieces_combine_to_the_whole_oracle(oracle_mod):
    w = synth.paired(scale=0.001)
    q, parts = 6, [0, 17, 42]
    whole = oracle_mod.count(w, restrict=(q, parts))
    wk, wc = whole.result()
    got = _oracle_par.count_restricted(w, q, parts, n_proc=2, piece_reads=1500)
    assert np.array_equal(got.keys, wk)
    assert np.array_equal(got.counts, wc)
    per = (w.bloom_bits // 64) >> q
    for p in parts:
        assert np.array_equal(got.words[p], whole.bloom(p * per, per))
    assert got.windows == whole.windows
    assert wk.size > 0
