"""Host-side bookkeeping of the combination technique (CPU only): the package's
layer set, layer weights and subdomain counts against the oracle's brute-force
enumeration and eq. Pchoice, and the total against the closed form that
precedes Table 1."""
import pytest

from oracle import combi
from paper_2110_11211_gb300 import combination


@pytest.mark.parametrize("d,L", [(1, 3), (2, 4), (2, 9), (3, 5), (3, 10), (4, 6), (4, 10),
                                 (5, 7), (6, 8)])
def test_layer_set_and_weights_match_the_oracle(d, L):
    ours = sorted((tuple(lv), combination.coefficient(d, i)) for lv, i in combination.layer_set(d, L))
    ref = sorted((tuple(lv), w) for lv, w in combi.full_layer_set(d, L))
    assert ours == ref
    # layer sizes: C(L + d - 2 - i, d - 1)
    for i in range(d):
        assert sum(1 for _, k in combination.layer_set(d, L) if k == i) == combi.layer_count(d, L, i)


@pytest.mark.parametrize("d,L,P_hat", [(2, 10, 4), (3, 10, 4), (4, 10, 4), (3, 12, 8)])
def test_subdomain_counts_follow_eq_pchoice(d, L, P_hat):
    from paper_2110_11211_gb300 import inputs
    total = 0
    for lv, i in combination.layer_set(d, L):
        n = inputs.grid_size(lv)
        P = combination.subdomain_count(d, i, P_hat, n)
        want = combi.subdomains_per_problem(d, i, P_hat)
        if 2 <= want <= n // 2:
            assert P == want, (lv, i)
        else:  # degenerate subgrids with few points keep 2 <= P <= N / 2
            assert 2 <= P <= max(2, n // 2), (lv, i, P)
        total += want
    assert total == combi.total_subdomains_closed_form(d, L, P_hat)
