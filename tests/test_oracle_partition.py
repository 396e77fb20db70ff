"""Pins for the partition, overlap, weights and coarse blocks
(eqs. sloc, enlarge, Di, omegai, restr; Lemma 3.1)."""
import numpy as np
import pytest

from oracle import partition as pt


@pytest.mark.parametrize("N,P", [(10, 3), (3969, 8), (221991, 128), (205065, 256), (64, 64)])
def test_tilde_sizes(N, P):
    s = pt.tilde_sizes(N, P)
    r = N % P
    assert s.sum() == N and s.size == P
    assert np.all(s[:r] == N // P + 1) and np.all(s[r:] == N // P)


@pytest.mark.parametrize("N,P,gamma", [(10, 3, 0.5), (37, 5, 0.2), (37, 5, 0.25), (50, 7, 1.0),
                                       (61, 9, 1.5), (61, 9, 2.0), (100, 11, 2.5), (23, 4, 0.75),
                                       (3969, 8, 0.5), (1000, 16, 0.3), (7, 2, 0.5)])
def test_ranges_match_set_definition(N, P, gamma):
    start, length = pt.overlap_ranges(N, P, gamma)
    sets = pt.overlap_sets_literal(N, P, gamma)
    for i in range(P):
        rng = set(pt.positions(start[i], length[i], N).tolist())
        assert rng == sets[i]
        assert len(rng) == length[i]  # no position repeated


@pytest.mark.parametrize("N,P,n", [(200, 5, 1), (200, 7, 2), (300, 9, 3), (3969, 8, 1), (1001, 12, 4)])
def test_lemma_half_integer_gamma(N, P, n):
    # Lemma 3.1: gamma = n/2 -> every point covered exactly 2 gamma + 1 times and
    # D_i = omega_i I = I / (2 gamma + 1).
    gamma = n / 2
    start, length = pt.overlap_ranges(N, P, gamma)
    cnt = pt.coverage_counts(N, start, length)
    assert np.all(cnt == n + 1)
    assert np.allclose(pt.omega_weights(N, start, length), 1.0 / (n + 1), rtol=0, atol=0)


def test_quarter_overlap_counts_and_weights():
    N, P = 205065, 256
    start, length = pt.overlap_ranges(N, P, 0.25)
    cnt = pt.coverage_counts(N, start, length)
    assert set(np.unique(cnt).tolist()) == {1, 2}
    assert np.all(pt.omega_weights(N, start, length) == 1.0)


def test_invalid_gamma_rejected():
    with pytest.raises(ValueError):
        pt.overlap_ranges(100, 3, 1.0)   # 2*1 + 1 = 3 = P
    with pytest.raises(ValueError):
        pt.overlap_ranges(100, 3, 0.0)


def test_coarse_blocks():
    for N, P, q in [(3969, 8, 16), (221991, 128, 64), (205065, 256, 32), (7, 2, 2), (10, 3, 3)]:
        bstart, bsize = pt.coarse_blocks(N, P, q)
        assert bsize.size == q * P
        # blocks tile [0, N) in order
        assert bstart[0] == 0 and np.array_equal(bstart[1:], np.cumsum(bsize)[:-1])
        assert bsize.sum() == N
        sizes = pt.tilde_sizes(N, P)
        offs = pt.tilde_offsets(sizes)
        for i in range(P):
            b = bsize[i * q:(i + 1) * q]
            assert bstart[i * q] == offs[i] and b.sum() == sizes[i]
            r = sizes[i] % q
            assert np.all(b[:r] == sizes[i] // q + 1) and np.all(b[r:] == sizes[i] // q)


def test_paper_q_rule():
    # four levels coarser: q = 2^{floor(log2 floor(N/P)) - 4}
    assert pt.paper_q(3969, 8) == 16
    assert pt.paper_q(221991, 128) == 64
    assert pt.paper_q(205065, 256) == 32
    assert pt.paper_q(4096575, 512) == 256
    assert pt.paper_q(256 * 64, 64) == 16   # S = 8 gives q = 2^{S-4}
    assert pt.paper_q(20, 4) == 1
