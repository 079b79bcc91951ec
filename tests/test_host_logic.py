"""Host logic of the library that needs no GPU: the solve server's memory
estimate, which admission under the device-memory budget relies on."""
import numpy as np

import instances as I
import paper_2609_02394_b300 as P


def test_estimate_grows_with_k_and_length():
    Js = list(np.random.default_rng(3).uniform(0.5, 1.5, 31))
    by_k = [P.estimate_bytes(I.xxz(32, Js, 1.0, 4, k, 8)) for k in (16, 32, 64, 128, 256)]
    assert all(a < b for a, b in zip(by_k, by_k[1:])), by_k
    by_n = [P.estimate_bytes(I.tfim(n, 1.0, 0.8, 4, 64, 4)) for n in (16, 32, 64, 128)]
    assert all(a <= b for a, b in zip(by_n, by_n[1:])), by_n


def test_estimate_covers_the_retained_blocks_and_fits_the_budget():
    c = I.rf_heisenberg_n128()                      # k = 256: the serving stream's largest requests
    est = P.estimate_bytes(c)
    # at least the Krylov-free floor: one merge's product-basis block of k_ret + 1
    # FP64 vectors of dimension k^2 (the retained basis it produces)
    assert est >= 8 * 257 * 256 * 256
    assert est < 40 << 30                           # admissible under the 40 GB serving budget


def test_estimate_rejects_a_bad_chain():
    c = I.tfim(8, 1.0, 0.8, 2, 8, 4)
    c.n_sites = 0
    assert P.estimate_bytes(c) == 0
