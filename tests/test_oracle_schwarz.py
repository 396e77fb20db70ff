"""Pins for the oracle's local/coarse operators, preconditioners and PCG
(Sec. 3.1, eqs. AS2a, csm, addSW, balSW; Lemma 3.1; Sec. 4 weak scaling)."""
import numpy as np
import pytest

from oracle import exact, grid, krylov, partition, schwarz


def dense_M(S, fn):
    N = S.N
    return np.column_stack([fn(np.eye(N)[:, k]) for k in range(N)])


def test_local_matrix_is_principal_submatrix():
    S = schwarz.Schwarz((3, 3), P=4, gamma=0.5)
    A = S.A.toarray()
    for i in range(S.P):
        ids = S.local_ids(i)
        R = np.zeros((ids.size, S.N))
        R[np.arange(ids.size), ids] = 1.0
        assert np.array_equal(S.local_matrix(i), R @ A @ R.T)


def test_coarse_matrix_one_dimensional_by_hand():
    # N = 7 (l = 3), P = 2 (tilde sizes 4, 3), q = 2: blocks {0,1},{2,3},{4,5},{6};
    # the 1-D curve is the identity, so A_0 = 64 * tridiag(-1, 2, -1) of size 4.
    S = schwarz.Schwarz((3,), P=2, gamma=0.5, q=2)
    T = 2 * np.eye(4) - np.eye(4, k=1) - np.eye(4, k=-1)
    assert np.array_equal(S.coarse_matrix(), 64.0 * T)


@pytest.mark.parametrize("levels,P,q,coeffs", [((3, 3), 4, 3, None), ((2, 3, 2), 5, 2, (1.0, 0.5, 2.0)),
                                               ((4, 4), 8, 4, None)])
def test_coarse_matrix_invariants(levels, P, q, coeffs):
    S = schwarz.Schwarz(levels, P=P, gamma=0.5, q=q, coeffs=coeffs)
    A0 = S.coarse_matrix()
    assert np.allclose(A0, A0.T, rtol=0, atol=1e-9)
    assert np.linalg.eigvalsh(A0).min() > 0
    # R_0^T 1 = 1 (blocks partition the grid) -> row sums of A_0 are block sums of A 1
    A1 = S.A @ np.ones(S.N)
    rs = np.array([A1[S.perm[s:s + n]].sum() for s, n in zip(S.bstart, S.bsize)])
    assert np.allclose(A0.sum(axis=1), rs, rtol=1e-13, atol=1e-9)


def test_singleton_coarse_blocks_give_exact_inverse():
    # q = N/P: every coarse block is one point, R_0 is a permutation and
    # F = R_0^T A_0^{-1} R_0 = A^{-1}.
    levels = (3, 2)                     # N = 21
    S = schwarz.Schwarz(levels, P=3, gamma=0.5, q=7)
    g = np.random.default_rng(0).standard_normal(S.N)
    assert np.allclose(S.coarse_correction(g), exact.solve(levels, g), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("levels,P,gamma,q", [((3, 3), 4, 0.5, 3), ((2, 2, 3), 6, 1.0, 2),
                                              ((4, 3), 5, 0.25, 4), ((3, 3), 4, 0.3, 2)])
def test_preconditioner_against_dense_definition(levels, P, gamma, q):
    """The index-slicing + Cholesky apply equals the definition built from the
    literal sets of eq. (enlarge) with dense selection matrices and explicit inverses."""
    S = schwarz.Schwarz(levels, P=P, gamma=gamma, q=q)
    A = S.A.toarray()
    N = S.N
    sets = partition.overlap_sets_literal(N, P, gamma)
    cnt = np.zeros(N)
    for s in sets:
        cnt[list(s)] += 1
    M = np.zeros((N, N))
    R0 = np.zeros((S.N0, N))
    for a, (s, n) in enumerate(zip(S.bstart, S.bsize)):
        R0[a, S.perm[s:s + n]] = 1.0
    M += R0.T @ np.linalg.inv(R0 @ A @ R0.T) @ R0
    for s in sets:
        pos = sorted(s)
        omega = max(1.0 / cnt[p] for p in pos)
        R = np.zeros((len(pos), N))
        R[np.arange(len(pos)), S.perm[pos]] = 1.0
        M += omega * R.T @ np.linalg.inv(R @ A @ R.T) @ R
    Mo = dense_M(S, S.apply)
    assert np.allclose(Mo, M, rtol=1e-10, atol=1e-12 * np.abs(M).max())


@pytest.mark.parametrize("variant", ["additive", "balanced"])
def test_preconditioner_symmetric_positive_definite(variant):
    S = schwarz.Schwarz((3, 3), P=5, gamma=0.5, q=2)
    fn = S.apply if variant == "additive" else S.apply_balanced
    M = dense_M(S, fn)
    assert np.allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_lemma_form_of_weighted_operator():
    # Lemma 3.1 consequence: gamma = 1/2 -> C_(2),D^{-1} = F + C_(1)^{-1} / 2
    S = schwarz.Schwarz((3, 4), P=6, gamma=0.5, q=2)
    g = np.random.default_rng(1).standard_normal(S.N)
    ref = S.coarse_correction(g) + 0.5 * S.one_level(g, weighted=False)
    assert np.allclose(S.apply(g), ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("levels,P,gamma", [((4, 4), 6, 0.5), ((3, 3, 2), 8, 1.0), ((5,), 4, 0.25)])
def test_pcg_reaches_exact_solution(levels, P, gamma):
    S = schwarz.Schwarz(levels, P=P, gamma=gamma)
    b = np.random.default_rng(2).uniform(-1, 1, S.N)
    x, its, hist = krylov.pcg(lambda v: S.A @ v, S.apply, b, rtol=1e-12)
    xe = exact.solve(levels, b)
    assert hist[-1] <= 1e-12
    assert np.linalg.norm(x - xe) <= 1e-9 * np.linalg.norm(xe)
    assert its < 60


def test_pcg_identity_and_exact_preconditioners():
    levels = (4, 3)
    A = grid.stencil_matrix(levels)
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    Ad = A.toarray()
    x, its, _ = krylov.pcg(lambda v: A @ v, lambda v: np.linalg.solve(Ad, v), b, rtol=1e-12)
    assert its == 1
    x, its, _ = krylov.pcg(lambda v: A @ v, lambda v: v.copy(), b, rtol=1e-10)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b) * 1.0001


def test_weak_scaling_iterations_bounded():
    """Sec. 4.1: with N/P and q fixed, the PCG iteration count reaches a constant
    as P grows, and the balanced variant needs about half the iterations of the
    additive one.  d = 1, N/P ~ 2^6, q = 2^{S-4} = 4, gamma = 1/2."""
    its, its_bal = [], []
    for P in (64, 128, 256):
        l = 6 + int(np.log2(P))
        S = schwarz.Schwarz((l,), P=P, gamma=0.5, q=4)
        b = np.random.default_rng(P).uniform(-1, 1, S.N)
        its.append(krylov.pcg(lambda v: S.A @ v, S.apply, b, rtol=1e-8)[1])
        its_bal.append(krylov.pcg(lambda v: S.A @ v, S.apply_balanced, b, rtol=1e-8)[1])
    assert max(its) <= 1.1 * min(its), its
    assert max(its_bal) <= 1.1 * min(its_bal), its_bal
    for k, kb in zip(its, its_bal):
        assert 0.4 <= kb / k <= 0.65, (its, its_bal)


def test_richardson_rate_bound():
    # eq. (redrate): with xi* the energy-norm error contracts by rho* = 1 - 2/(1+kappa)
    S = schwarz.Schwarz((4, 4), P=4, gamma=0.5, q=2)
    A = S.A.toarray()
    M = dense_M(S, S.apply)
    ev = np.sort(np.linalg.eigvals(M @ A).real)
    lmin, lmax = ev[0], ev[-1]
    xi = 2.0 / (lmin + lmax)
    rho = 1.0 - 2.0 / (1.0 + lmax / lmin)
    x0 = np.random.default_rng(6).uniform(-1, 1, S.N)
    enorm = lambda v: float(np.sqrt(v @ (A @ v)))
    x = x0.copy()
    for k in range(1, 11):
        x = x + xi * S.apply(-(A @ x))      # f = 0: the iterate is the error
        assert enorm(x) <= rho ** k * enorm(x0) * (1 + 1e-9)


@pytest.mark.parametrize("levels,P,gamma,q,weighting", [((3, 3), 4, 0.5, 3, "omega"),
                                                        ((2, 2, 3), 6, 1.0, 2, "omega"),
                                                        ((4, 3), 5, 0.25, 4, "omega"),
                                                        ((3, 3), 5, 0.5, 2, "none")])
def test_balanced_operator_against_dense_definition(levels, P, gamma, q, weighting):
    """eq. (balan) / (balSW) built from dense matrices: F = R_0^T A_0^{-1} R_0
    with R_0 from the blocks of eq. (restr), C_(1),D^{-1} = sum_i omega_i R_i^T
    A_i^{-1} R_i from the literal sets of eq. (enlarge), G = I - A F and
    M = G^T C_(1),D^{-1} G + F with G^T formed by an explicit transpose.  A
    swap of G and G^T gives G C G^T + F, also symmetric positive definite, but
    another matrix: it is checked to differ."""
    S = schwarz.Schwarz(levels, P=P, gamma=gamma, q=q, weighting=weighting)
    A = S.A.toarray()
    N = S.N
    sets = partition.overlap_sets_literal(N, P, gamma)
    cnt = np.zeros(N)
    for s in sets:
        cnt[list(s)] += 1
    R0 = np.zeros((S.N0, N))
    for a, (s, n) in enumerate(zip(S.bstart, S.bsize)):
        R0[a, S.perm[s:s + n]] = 1.0
    F = R0.T @ np.linalg.inv(R0 @ A @ R0.T) @ R0
    C1 = np.zeros((N, N))
    for s in sets:
        pos = sorted(s)
        omega = max(1.0 / cnt[p] for p in pos) if weighting == "omega" else 1.0
        R = np.zeros((len(pos), N))
        R[np.arange(len(pos)), S.perm[pos]] = 1.0
        C1 += omega * R.T @ np.linalg.inv(R @ A @ R.T) @ R
    G = np.eye(N) - A @ F
    M = G.T @ C1 @ G + F
    Mo = dense_M(S, S.apply_balanced)
    assert np.allclose(Mo, M, rtol=1e-10, atol=1e-11 * np.abs(M).max())
    swapped = G @ C1 @ G.T + F
    assert np.abs(swapped - M).max() > 1e-3 * np.abs(M).max()
