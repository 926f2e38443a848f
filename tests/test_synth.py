"""The seeded input generators: pieces of a record join into the same record."""
import numpy as np

import synth


def test_parallel_adc_generator_equals_the_sequential_one():
    # the bench builds long int16 records piecewise in a process pool; the pieces
    # must join into exactly the record the sequential generator produces
    n = 3 * (1 << 14) + 123
    seq, _ = synth.adc_telegraph_int16(n, seed=9, p=2e-3)
    par = synth.adc_telegraph_int16_parallel(n, seed=9, p=2e-3, piece=1 << 14, processes=2)
    assert par.dtype == np.int16
    assert np.array_equal(seq, par)


def test_piecewise_adc_generator_equals_one_call():
    n = 5000
    one, _ = synth.adc_telegraph_int16(n, seed=4, p=1e-2)
    a, st = synth.adc_telegraph_int16(1234, seed=4, p=1e-2)
    b, _ = synth.adc_telegraph_int16(n - 1234, seed=4, start=1234, state=st, p=1e-2)
    assert np.array_equal(one, np.concatenate([a, b]))
