"""The coarse table's claim, pinned on the oracle (no GPU): a super-bin of f
adjacent bins, whose window is the union of the members' windows, has exactly
the OR of the members' bit vectors (every q-gram of the union lies wholly in
one member window because ext >= q-1), so its token sum bounds every
member's sum from above and a super-bin below the threshold rules out all of
its members."""
import numpy as np
import pytest

import oracle
from tests.conftest import Reads, random_case

@pytest.mark.parametrize("F", [2, 3, 5])
@pytest.mark.parametrize("seed", range(6))
def test_super_bin_vector_is_or_of_members(seed, F):
    rng = np.random.default_rng(40 + seed)
    q = int(rng.choice([2, 3, 4, 5]))
    B = int(rng.integers(3, 50))
    mrl = int(rng.integers(q, 60))
    n = int(rng.integers(100, 5000))
    ref, _, _ = random_case(rng, q, n, B, mrl, 0)
    g = np.frombuffer(ref.encode(), np.uint8)
    fine = oracle.bin_vectors(g, B, q, mrl)
    coarse = oracle.bin_vectors(g, F * B, q, mrl)
    assert coarse.num_bins == -(-fine.num_bins // F)
    for s in range(coarse.num_bins):
        members = fine.vecs[F * s: F * s + F]
        assert np.array_equal(coarse.vecs[s], np.bitwise_or.reduce(members, axis=0)), s


@pytest.mark.parametrize("F", [2, 4])
@pytest.mark.parametrize("seed", range(4))
def test_super_bin_sum_bounds_member_sums(seed, F):
    rng = np.random.default_rng(60 + seed)
    q = int(rng.choice([3, 4, 5]))
    B = int(rng.integers(5, 40))
    mrl = int(rng.integers(max(q, 10), 50))
    ref, reads, e = random_case(rng, q, 3000, B, mrl, 40)
    g = np.frombuffer(ref.encode(), np.uint8)
    fine = oracle.bin_vectors(g, B, q, mrl)
    coarse = oracle.bin_vectors(g, F * B, q, mrl)
    rs = Reads(reads, [60] * len(reads))  # T <= 0: every sum is reported
    fr, fb, fc = oracle.filter(fine, rs)
    cr, cb, cc = oracle.filter(coarse, rs)
    fsum = np.zeros((len(reads), fine.num_bins), np.int64)
    csum = np.zeros((len(reads), coarse.num_bins), np.int64)
    fsum[fr, fb] = fc
    csum[cr, cb] = cc
    for k in range(F):
        members = np.arange(k, fine.num_bins, F)
        assert (csum[:, members // F] >= fsum[:, members]).all()
