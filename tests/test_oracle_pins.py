"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test would fail under a plausible mistake in the oracle: a swapped
parity, a wrong index set in Algorithm 2, a transposed block, a dropped
boundary term, a wrong sign or a wrong normalisation.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


def chain_from_T(A, m=1):
    """Oracle chain whose T = Q^T equals the given block-tridiagonal A."""
    N = A.shape[0]
    L = N // m
    Q = A.T
    dn = np.zeros((L, m, m)); loc = np.zeros((L, m, m)); up = np.zeros((L, m, m))
    for l in range(L):
        s = slice(l * m, (l + 1) * m)
        loc[l] = Q[s, s]
        if l > 0:
            dn[l] = Q[s, (l - 1) * m:l * m]
        if l < L - 1:
            up[l] = Q[s, (l + 1) * m:(l + 2) * m]
    return oracle.Chain(dn, loc, up)


def spectrum(G):
    ev = np.linalg.eigvals(G)
    return np.array(sorted(ev, key=lambda z: (round(z.real, 9), round(z.imag, 9))))


def same_multiset(ev, ref, tol=1e-12):
    ev = list(ev)
    for r in ref:
        k = int(np.argmin([abs(e - r) for e in ev]))
        if abs(ev[k] - r) > tol:
            return False
        ev.pop(k)
    return not ev


# --- Sect. 2, Examples 1 and 2 -------------------------------------------------

def test_example1_and_2_spectra():
    g = read_golden("example1_2.txt")
    A = np.array(g["matrix"])
    ch = chain_from_T(A)
    assert np.array_equal(ch.dense_T(), A)
    assert same_multiset(np.linalg.eigvals(ch.iteration_matrix(oracle.BJ)), g["jacobi"][0])
    assert same_multiset(np.linalg.eigvals(ch.iteration_matrix(oracle.BGS)), g["gauss_seidel"][0])
    assert same_multiset(np.linalg.eigvals(ch.iteration_matrix(oracle.STAIR1)), g["stair1"][0])
    # the transposed matrix has the same spectra (the paper's matrix has zero
    # row sums, i.e. it is really Q; reading it as Q^T or Q gives one answer)
    chT = chain_from_T(A.T.copy())
    assert same_multiset(np.linalg.eigvals(chT.iteration_matrix(oracle.STAIR1)), g["stair1"][0])


def test_example2_pins_index_set_reading():
    """Algorithm 2 step 1 read literally (k = i included for coupled rows)
    does NOT give Example 2's spectrum; the reading with k != i does."""
    g = read_golden("example1_2.txt")
    A = np.array(g["matrix"])
    n = 4
    # literal reading, 1-based rows: odd rows J={i}; even rows J={i-1,i+1}
    G = np.zeros((n, n))
    for c in range(n):
        x = np.zeros(n); x[c] = 1.0
        z = np.zeros(n)
        for i in range(1, n + 1):
            J = {i} if i % 2 == 1 else {i - 1, i + 1} & set(range(1, n + 1))
            z[i - 1] = -sum(A[i - 1, k - 1] * x[k - 1] for k in range(1, n + 1) if k not in J)
        for i in range(1, n + 1, 2):
            z[i - 1] = z[i - 1] / A[i - 1, i - 1]
        for i in range(2, n + 1, 2):
            J = {i - 1, i + 1} & set(range(1, n + 1))
            z[i - 1] = (z[i - 1] - sum(A[i - 1, k - 1] * z[k - 1] for k in J)) / A[i - 1, i - 1]
        G[:, c] = z
    assert not same_multiset(np.linalg.eigvals(G), g["stair1"][0], tol=1e-6)
    ours = chain_from_T(A).iteration_matrix(oracle.STAIR1)
    assert same_multiset(np.linalg.eigvals(ours), g["stair1"][0])


# --- splittings against explicitly assembled M, N ----------------------------

def stair_M(T, L, m, typ):
    """Stair matrix of type 1 or 2 assembled from dense T (Sect. 2)."""
    M = np.zeros_like(T)
    for l in range(L):
        s = slice(l * m, (l + 1) * m)
        M[s, s] = T[s, s]
        one_based_odd = (l + 1) % 2 == 1
        coupled = (not one_based_odd) if typ == 1 else one_based_odd
        if coupled:
            if l > 0:
                M[s, (l - 1) * m:l * m] = T[s, (l - 1) * m:l * m]
            if l < L - 1:
                M[s, (l + 1) * m:(l + 2) * m] = T[s, (l + 1) * m:(l + 2) * m]
    return M


def bgs_M(T, L, m):
    M = np.zeros_like(T)
    for l in range(L):
        M[l * m:(l + 1) * m, :(l + 1) * m] = T[l * m:(l + 1) * m, :(l + 1) * m]
    return M


def bj_M(T, L, m):
    M = np.zeros_like(T)
    for l in range(L):
        s = slice(l * m, (l + 1) * m)
        M[s, s] = T[s, s]
    return M


def dense_QT(dn, loc, up):
    """Q^T assembled straight from the generator blocks (independent of the oracle)."""
    L, m, _ = loc.shape
    Q = np.zeros((L * m, L * m))
    for l in range(L):
        Q[l * m:(l + 1) * m, l * m:(l + 1) * m] = loc[l]
        if l > 0:
            Q[l * m:(l + 1) * m, (l - 1) * m:l * m] = dn[l]
        if l < L - 1:
            Q[l * m:(l + 1) * m, (l + 1) * m:(l + 2) * m] = up[l]
    return Q.T.copy()


@pytest.mark.parametrize("L,m", [(7, 3), (8, 4), (2, 5), (3, 1), (9, 2)])
def test_sweeps_equal_dense_splittings(L, m):
    dn, loc, up = synth.qbd(L, m, 0.8, seed=21 + L, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    T = dense_QT(dn, loc, up)
    assert np.allclose(ch.dense_T(), T, rtol=0, atol=0)
    x = np.random.default_rng(L * 100 + m).random(L * m)
    for meth, M in [(oracle.STAIR1, stair_M(T, L, m, 1)), (oracle.STAIR2, stair_M(T, L, m, 2)),
                    (oracle.BGS, bgs_M(T, L, m)), (oracle.BJ, bj_M(T, L, m))]:
        N = M - T
        ref = np.linalg.solve(M, N @ x)
        z = ch.sweep(x, meth)
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max(), meth


@pytest.mark.parametrize("L,m", [(7, 3), (11, 6)])
@pytest.mark.parametrize("meth", [oracle.STAIR1, oracle.STAIR2, oracle.BGS, oracle.BJ])
def test_normalised_sweep_equals_dense_step(L, m, meth):
    """One step of Eq. (2) (the expected [e^T z, step] of every GPU stats
    check): z = M^{-1} N x from independently assembled M and N, s = e^T z,
    pi = z / s, and the step error ||pi - x||_1 against the normalised pi.
    x is a unit-L1 vector far from equilibrium, so s differs from 1 and a
    step error taken against the unnormalised z, or s summed over x, fails."""
    dn, loc, up = synth.qbd(L, m, 0.8, seed=50 + L * m, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    T = dense_QT(dn, loc, up)
    M = {oracle.STAIR1: stair_M(T, L, m, 1), oracle.STAIR2: stair_M(T, L, m, 2),
         oracle.BGS: bgs_M(T, L, m), oracle.BJ: bj_M(T, L, m)}[meth]
    x = np.random.default_rng(L + 7 * m).random(L * m) ** 4
    x /= x.sum()
    z = np.linalg.solve(M, (M - T) @ x)
    s_ref = z.sum()
    pi_ref = z / s_ref
    d_ref = np.abs(pi_ref - x).sum()
    pi, s, d = ch.normalised_sweep(x, meth)
    assert abs(s - s_ref) <= 1e-14 * abs(s_ref)
    assert np.abs(pi - pi_ref).sum() <= 1e-14 * np.abs(pi_ref).sum()
    assert abs(d - d_ref) <= 1e-14
    assert abs(s_ref - 1.0) > 1e-3 and abs(np.abs(z - x).sum() - d_ref) > 1e-6
    assert abs(x.sum() - s_ref) > 1e-3


@pytest.mark.parametrize("L,m", [(7, 3), (8, 4), (5, 1)])
def test_sweep_with_rhs_equals_dense(L, m):
    """The refinement step z = M^{-1}(N x + b), against dense M and N."""
    dn, loc, up = synth.qbd(L, m, 0.8, seed=40 + L, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    T = dense_QT(dn, loc, up)
    rng = np.random.default_rng(L)
    x = rng.random(L * m)
    b = rng.standard_normal(L * m)
    for meth, M in [(oracle.STAIR1, stair_M(T, L, m, 1)), (oracle.STAIR2, stair_M(T, L, m, 2)),
                    (oracle.BGS, bgs_M(T, L, m)), (oracle.BJ, bj_M(T, L, m))]:
        ref = np.linalg.solve(M, (M - T) @ x + b)
        z = ch.sweep_rhs(x, b, meth)
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max(), meth
        assert np.array_equal(ch.sweep_rhs(x, np.zeros_like(b), meth), ch.sweep(x, meth))
    assert np.allclose(ch.residual_vec(x), T @ x, rtol=1e-14, atol=1e-15)


def test_refinement_fixed_point_solves_correction_equation():
    """Iterating z = M^{-1}(N d - r) drives T d + r to zero (e^T r = 0)."""
    dn, loc, up = synth.qbd(10, 3, 0.8, seed=2, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    pi = np.full(30, 1 / 30)
    r = ch.residual_vec(pi)
    assert abs(r.sum()) < 1e-15
    d = np.zeros(30)
    for _ in range(3000):
        d = ch.sweep_rhs(d, -r)
    T = dense_QT(dn, loc, up)
    assert np.abs(T @ d + r).sum() <= 1e-12
    x = (pi + d) / (pi + d).sum()
    ref = direct_pi(dn, loc, up)
    assert np.abs(x - ref).sum() <= 1e-11


def test_residual_against_dense():
    dn, loc, up = synth.qbd(9, 4, 0.8, seed=4, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    x = np.random.default_rng(0).random(36)
    ref = np.abs(dense_QT(dn, loc, up) @ x).sum()
    assert abs(ch.residual(x) - ref) <= 1e-13 * ref


@pytest.mark.parametrize("method,coupled_parity", [(oracle.STAIR1, 1), (oracle.STAIR2, 0)])
def test_stair_sweep_zeroes_the_coupled_rows_of_the_residual(method, coupled_parity):
    """With M the stair matrix, M z = N x holds row by row; on the coupled
    (half-sweep-2) block rows M and T agree (N is zero there), so Q^T z = 0
    on those rows, while on the diagonal-only rows Q^T z = N (x - z)."""
    L, m = 11, 6
    dn, loc, up = synth.qbd(L, m, 0.85, seed=12, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    x = np.random.default_rng(3).random(L * m)
    z = ch.sweep(x, method)
    r = ch.residual_vec(z).reshape(L, m)
    scale = np.abs(z).max() * np.abs(dense_QT(dn, loc, up)).max()
    coupled = np.arange(L) % 2 == coupled_parity
    assert np.abs(r[coupled]).max() <= 1e-13 * scale
    # the diagonal-only rows carry the whole residual: N (x - z) there
    T = dense_QT(dn, loc, up)
    N = np.zeros_like(T)
    for l in np.nonzero(~coupled)[0]:
        s = slice(l * m, (l + 1) * m)
        N[s] = -T[s]
        N[s, s] = 0.0
    ref = (N @ (x - z)).reshape(L, m)
    assert np.abs(r[~coupled] - ref[~coupled]).max() <= 1e-12 * scale
    assert np.abs(r[~coupled]).max() > 1e-6 * scale     # not trivially zero


# --- LU --------------------------------------------------------------------------

def test_lu_reconstruction_no_swaps_on_diag_blocks():
    dn, loc, up = synth.qbd(20, 16, 0.9, seed=9, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    assert ch.swaps == 0          # column-diagonally dominant blocks
    for l in range(ch.L):
        LU = ch.LU[l]
        Lm = np.tril(LU, -1) + np.eye(ch.m)
        Um = np.triu(LU)
        err = np.abs(Lm @ Um - ch.Tdd[l]).max()
        assert err <= 1e-14 * np.abs(ch.Tdd[l]).max() * ch.m


def test_lu_partial_pivoting_general_matrix():
    import ctypes
    rng = np.random.default_rng(5)
    m = 9
    A = rng.standard_normal((m, m))
    LU = A.copy()
    piv = np.zeros(m, np.int32)
    lib = oracle._load()
    swaps = lib.or_lu(m, ctypes.c_void_p(LU.ctypes.data), ctypes.c_void_p(piv.ctypes.data))
    assert swaps > 0
    P = np.eye(m)
    for k in range(m):
        P[[k, piv[k]]] = P[[piv[k], k]]
    Lm = np.tril(LU, -1) + np.eye(m)
    assert np.abs(P @ A - Lm @ np.triu(LU)).max() < 1e-13
    assert np.abs(np.tril(LU, -1)).max() <= 1.0 + 1e-15      # |l_ik| <= 1
    b = rng.standard_normal(m)
    x = b.copy()
    lib.or_lu_solve(m, ctypes.c_void_p(LU.ctypes.data), ctypes.c_void_p(piv.ctypes.data),
                    ctypes.c_void_p(x.ctypes.data))
    assert np.abs(A @ x - b).max() < 1e-12
    Z = np.zeros((m, m)); Z[:, 0] = 1.0
    assert lib.or_lu(m, ctypes.c_void_p(Z.ctypes.data), ctypes.c_void_p(piv.ctypes.data)) == -1


# --- the limit pi ------------------------------------------------------------------

def direct_pi(dn, loc, up):
    """Dense direct solve of Q^T pi = 0 with one equation replaced by e^T pi = 1."""
    T = dense_QT(dn, loc, up)
    T[-1, :] = 1.0
    b = np.zeros(T.shape[0]); b[-1] = 1.0
    return np.linalg.solve(T, b)


@pytest.mark.parametrize("L,m,dep", [(6, 3, True), (11, 4, True), (64, 8, False), (5, 1, True)])
def test_limit_matches_dense_direct_solve(L, m, dep):
    dn, loc, up = synth.qbd(L, m, 0.8, seed=L + m, level_dependent=dep)
    ch = oracle.Chain(dn, loc, up)
    res = ch.solve(tol=1e-14, maxit=200000, check_every=10)
    pi = res["x"]
    ref = direct_pi(dn, loc, up)
    assert np.abs(pi - ref).sum() / np.abs(ref).sum() <= 1e-11
    assert (pi >= 0).all() and abs(pi.sum() - 1.0) <= 1e-14
    assert res["resid"] <= 1e-14


def test_birth_death_closed_form():
    L, lam, mu = 64, 0.8, 1.0
    ch = oracle.Chain(*synth.birth_death(L, lam, mu))
    res = ch.solve(tol=1e-15, maxit=100000, check_every=10)
    r = lam / mu
    ref = (1 - r) * r ** np.arange(L) / (1 - r ** L)
    assert np.abs(res["x"] - ref).sum() / ref.sum() <= 1e-11
    # the residual of the exact closed form is at the rounding floor
    assert ch.residual(ref) <= 1e-15


def test_stopping_rule_step_error():
    dn, loc, up = synth.qbd(16, 4, 0.8, seed=1, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    res = ch.solve(tol=0.0, eps=1e-9, maxit=100000)
    h = res["hist"]
    assert h[-1] <= 1e-9 < h[-2]
    res2 = ch.solve(tol=0.0, eps=0.0, maxit=37)
    assert res2["sweeps"] == 37


def test_breakdown_detected():
    dn, loc, up = synth.qbd(6, 2, 0.8, seed=1, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    with pytest.raises(FloatingPointError):
        ch.solve(x0=-np.ones(12) / 12, maxit=5)


# --- convergence rate (Sect. 2, feature 2) ------------------------------------------

def second_eig(G):
    ev = np.linalg.eigvals(G)
    ev = ev[np.argsort(-np.abs(ev))]
    assert abs(ev[0] - 1.0) < 1e-10
    return abs(ev[1])


@pytest.mark.parametrize("L,m,seed", [(8, 3, 1), (10, 4, 2), (7, 5, 3)])
def test_stair_bgs_same_spectrum_and_young(L, m, seed):
    dn, loc, up = synth.qbd(L, m, 0.8, seed=seed, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    G1 = ch.iteration_matrix(oracle.STAIR1)
    G2 = ch.iteration_matrix(oracle.STAIR2)
    Gg = ch.iteration_matrix(oracle.BGS)
    Gj = ch.iteration_matrix(oracle.BJ)
    # eigenvalues near 0 sit in Jordan blocks and are ill-conditioned; the
    # well-separated part of the spectrum (|lambda| > 0.05) must coincide
    def big(G):
        e = np.sort(np.abs(np.linalg.eigvals(G)))
        return e[e > 0.05]
    e1, e2, eg = big(G1), big(G2), big(Gg)
    assert len(e1) == len(eg) == len(e2) and len(eg) >= L // 2
    assert np.abs(e1 - eg).max() <= 1e-9 and np.abs(e2 - eg).max() <= 1e-9
    ej = np.linalg.eigvals(Gj)
    # block Jacobi on a bipartite level graph: -1 is an eigenvalue too
    assert np.min(np.abs(ej + 1.0)) < 1e-9
    gj = np.sort(np.abs(ej))[-3]           # largest modulus other than +-1
    assert abs(second_eig(Gg) - gj ** 2) <= 1e-9


@pytest.mark.slow
def test_observed_contraction_equals_bgs_and_eigenvalue():
    dn, loc, up = synth.workload("qbd_L64_m8")
    ch = oracle.Chain(dn, loc, up)
    gamma = second_eig(ch.iteration_matrix(oracle.STAIR1))
    r1 = ch.solve(tol=0.0, eps=1e-14, maxit=20000)
    rg = ch.solve(tol=0.0, eps=1e-14, maxit=20000, method=oracle.BGS)
    # asymptotic regime: a window before the rounding floor
    k1 = oracle.contraction(r1["hist"][: int(0.8 * len(r1["hist"]))], 200)
    kg = oracle.contraction(rg["hist"][: int(0.8 * len(rg["hist"]))], 200)
    assert abs(k1 - kg) < 1e-3
    assert abs(k1 - gamma) < 1e-3
    # block Jacobi does not converge (|lambda| = 1 twice)
    rj = ch.solve(tol=0.0, eps=1e-14, maxit=400, method=oracle.BJ)
    assert rj["sweeps"] == 400 and rj["step"] > 1e-6


# --- block-banded Q^T: Algorithm 2 with off-staircase terms |k - i| >= 2 --------------

def banded_dense_QT(D, L, m):
    Q = np.zeros((L * m, L * m))
    for e, B in D.items():
        for l in range(L):
            k = l + e
            if 0 <= k < L:
                Q[l * m:(l + 1) * m, k * m:(k + 1) * m] = B[l]
    return Q.T.copy()


@pytest.mark.parametrize("L,m,p,q", [(9, 3, 1, 3), (10, 2, 2, 2), (8, 4, 3, 1), (7, 1, 2, 3)])
def test_banded_sweeps_equal_dense_splittings(L, m, p, q):
    D = synth.banded(L, m, p, q, 0.8, seed=L + 10 * p + q)
    bc = oracle.BandedChain(D)
    T = banded_dense_QT(D, L, m)
    assert np.array_equal(bc.dense_T(), T)
    x = np.random.default_rng(L).random(L * m)
    for meth, M in [(oracle.STAIR1, stair_M(T, L, m, 1)), (oracle.STAIR2, stair_M(T, L, m, 2)),
                    (oracle.BGS, bgs_M(T, L, m)), (oracle.BJ, bj_M(T, L, m))]:
        ref = np.linalg.solve(M, (M - T) @ x)
        z = bc.sweep(x, meth)
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max(), meth
    assert abs(bc.residual(x) - np.abs(T @ x).sum()) <= 1e-13 * np.abs(T @ x).sum()


def test_banded_reduces_to_tridiagonal_oracle():
    dn, loc, up = synth.qbd(12, 4, 0.8, seed=2, level_dependent=True)
    bc = oracle.BandedChain({-1: dn, 0: loc, 1: up})
    ch = oracle.Chain(dn, loc, up)
    x = np.random.default_rng(3).random(48)
    for meth in (oracle.STAIR1, oracle.STAIR2, oracle.BGS, oracle.BJ):
        assert np.allclose(bc.sweep(x, meth), ch.sweep(x, meth), rtol=1e-14, atol=0)


def test_banded_limit_matches_direct_solve():
    L, m = 14, 3
    D = synth.banded(L, m, 1, 3, 0.7, seed=4)
    bc = oracle.BandedChain(D)
    res = bc.solve(tol=1e-14, maxit=200000, check_every=20)
    T = banded_dense_QT(D, L, m)
    T[-1, :] = 1.0
    b = np.zeros(L * m); b[-1] = 1.0
    ref = np.linalg.solve(T, b)
    assert np.abs(res["x"] - ref).sum() <= 1e-11 and res["resid"] <= 1e-14


def test_block_hessenberg_stair_rate_close_to_gauss_seidel():
    """Sect. 2 / Example 3: on block Hessenberg singular M-matrices the staircase
    spectral gap stays close to block Gauss-Seidel's (rho_2 near 1)."""
    D = synth.banded(10, 3, 1, 3, 0.8, seed=7)
    bc = oracle.BandedChain(D)

    def gamma(meth):
        G = np.empty((bc.N, bc.N))
        for k in range(bc.N):
            e = np.zeros(bc.N); e[k] = 1.0
            G[:, k] = bc.sweep(e, meth)
        ev = np.sort(np.abs(np.linalg.eigvals(G)))
        assert abs(ev[-1] - 1.0) < 1e-9
        return ev[-2]
    g_bs, g_bgs = gamma(oracle.STAIR1), gamma(oracle.BGS)
    rho2 = np.log(1 / g_bgs) / np.log(1 / g_bs)
    assert 0.5 < rho2 < 2.0


# --- mixed-precision storage and the refinement step --------------------------------

def test_round_bf16_ties_and_torch():
    """BF16 keeps 8 significant bits, rounding to nearest with ties to even."""
    r = oracle.round_bf16
    one = 1.0
    assert r(one + 2.0 ** -8) == 1.0                 # tie, 1.0 is even
    assert r(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie, rounds to the even neighbour
    assert r(one + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert r(-(one + 3 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)
    assert r(0.0) == 0.0 and r(0.75) == 0.75
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(4).standard_normal(20000).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(r(x), ref)


def test_quantize_block_scale_and_grid():
    rng = np.random.default_rng(9)
    B = rng.random((16, 16)) * 37.0
    Q = oracle.quantize_block(B, "bf16")
    e = int(np.frexp(np.abs(B).max())[1])
    S = Q / 2.0 ** e
    assert 0.5 <= np.abs(S).max() <= 1.0                        # scale from the block max
    assert np.array_equal(oracle.round_bf16(S), S)              # mantissas on the BF16 grid
    assert np.abs(Q - B).max() <= 2.0 ** -9 * 2.0 ** e          # half a BF16 ulp at the top
    assert np.array_equal(oracle.quantize_block(B, "f32"), B.astype(np.float32).astype(np.float64))
    assert np.array_equal(oracle.quantize_block(np.zeros((3, 3)), "bf16"), np.zeros((3, 3)))


@pytest.mark.parametrize("apply", ["inverse", "coupled"])
@pytest.mark.parametrize("method", [oracle.STAIR1, oracle.STAIR2])
def test_refinement_step_fp64_equals_correction_sweeps(apply, method):
    """Without quantization the refinement step is K correction sweeps
    z = M^{-1}(N z - r) from zero (the pinned or_sweep_rhs), then the
    renormalised pi0 + z; the explicit inverse and the coupled operators give
    the LU solves' values up to rounding."""
    L, m, K = 9, 6, 7
    dn, loc, up = synth.qbd(L, m, 0.85, seed=70, level_dependent=True)
    ch = oracle.Chain(dn, loc, up)
    pi0 = np.random.default_rng(2).random(L * m)
    pi0 /= pi0.sum()
    r = ch.residual_vec(pi0)
    d = np.zeros(L * m)
    for _ in range(K):
        d = ch.sweep_rhs(d, -r, method)
    ref = (pi0 + d) / (pi0 + d).sum()
    got = ch.refinement_step(pi0, K, "f64", apply, method)
    assert np.abs(got - ref).sum() <= 1e-13 * np.abs(ref).sum()
    # low-precision storage moves the step by its rounding only
    for dtype, tol in (("f32", 1e-6), ("bf16", 2e-2)):
        q = ch.refinement_step(pi0, K, dtype, apply, method)
        err = np.abs(q - ref).sum() / np.abs(ref).sum()
        assert 0.0 < err <= tol, (dtype, err)
