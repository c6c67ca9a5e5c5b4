"""Generator synthesiser: structural properties of the synthetic generators."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import synth


def dense_Q(dn, loc, up):
    L, m, _ = loc.shape
    Q = np.zeros((L * m, L * m))
    for l in range(L):
        Q[l * m:(l + 1) * m, l * m:(l + 1) * m] = loc[l]
        if l > 0:
            Q[l * m:(l + 1) * m, (l - 1) * m:l * m] = dn[l]
        if l < L - 1:
            Q[l * m:(l + 1) * m, (l + 1) * m:(l + 2) * m] = up[l]
    return Q


@pytest.mark.parametrize("L,m,ratio,dep", [(64, 8, 0.8, False), (37, 5, 0.9, True), (2, 3, 0.7, True)])
def test_qbd_is_a_generator(L, m, ratio, dep):
    dn, loc, up = synth.qbd(L, m, ratio, seed=11, level_dependent=dep)
    Q = dense_Q(dn, loc, up)
    off = Q - np.diag(np.diag(Q))
    assert (off >= 0).all()
    assert (np.diag(Q) < 0).all()
    assert np.abs(Q.sum(1)).max() <= 1e-13 * np.abs(Q).max() * m
    assert not dn[0].any() and not up[L - 1].any()
    # diagonals of A0 / A2 forced positive where retained
    for l in range(L):
        if l < L - 1:
            assert (np.diag(up[l]) > 0).all()
        if l > 0:
            assert (np.diag(dn[l]) > 0).all()
    # irreducible: the state graph is strongly connected
    n, _ = connected_components(sp.csr_matrix(off > 0), directed=True, connection="strong")
    assert n == 1


def test_qbd_up_down_ratio_and_values():
    L, m, ratio = 40, 6, 0.85
    dn, loc, up = synth.qbd(L, m, ratio, seed=3, level_dependent=True)
    for l in range(1, L - 1):
        assert abs(up[l].sum() / dn[l].sum() - ratio) <= 1e-14
    nz = up[1:-1][up[1:-1] > 0]
    assert nz.min() >= 0.1 and nz.max() < 1.0
    # off-diagonal density of A0 is about 1/2 (diagonal forced)
    offd = up[:-1].copy()
    for l in range(L - 1):
        np.fill_diagonal(offd[l], 0)
    frac = (offd > 0).sum() / ((L - 1) * m * (m - 1))
    assert 0.4 < frac < 0.6
    # level dependence: distinct levels differ; level independence: equal
    assert not np.array_equal(up[1], up[2])
    dn2, loc2, up2 = synth.qbd(L, m, ratio, seed=3, level_dependent=False)
    assert np.array_equal(up2[1], up2[2]) and np.array_equal(loc2[3], loc2[7])


def test_qbd_bitwise_deterministic_and_subrange():
    a = synth.qbd(50, 7, 0.9, seed=5, level_dependent=True)
    b = synth.qbd(50, 7, 0.9, seed=5, level_dependent=True)
    c = synth.qbd(50, 7, 0.9, seed=5, level_dependent=True, l0=13, l1=29)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y)
        assert np.array_equal(x[13:29], z)
    d = synth.qbd(50, 7, 0.9, seed=6, level_dependent=True)
    assert not np.array_equal(a[1], d[1])


def test_penta_paired_structure():
    L, m = 12, 3
    dn, loc, up = synth.penta_paired(L, m, 0.8, 0.3, seed=2)
    assert loc.shape == (L // 2, 2 * m, 2 * m)
    Q = dense_Q(dn, loc, up)
    assert np.abs(Q.sum(1)).max() <= 1e-14 * np.abs(Q).max() * m
    off = Q - np.diag(np.diag(Q))
    assert (off >= 0).all()
    # structurally zero quadrants of the paired off-diagonal blocks
    for J in range(1, L // 2 - 1):
        assert not up[J][:m, m:].any()      # level 2J -> 2J+3
        assert not dn[J][m:, :m].any()      # level 2J+1 -> 2J-2
    # unpaired view: jumps only to levels within distance 2
    N = L * m
    lev = np.arange(N) // m
    i, j = np.nonzero(off)
    assert np.abs(lev[i] - lev[j]).max() == 2
    # up/down rate ratio of interior levels (rate sums, size-2 jumps scaled 0.3)
    l = 4
    rows = slice(l * m, (l + 1) * m)
    upr = sum(off[rows, k * m:(k + 1) * m].sum() for k in (l + 1, l + 2))
    dnr = sum(off[rows, k * m:(k + 1) * m].sum() for k in (l - 1, l - 2))
    assert abs(upr / dnr - 0.8) < 1e-13


def test_birth_death_blocks():
    dn, loc, up = synth.birth_death(10, 0.8, 1.0)
    Q = dense_Q(dn, loc, up)
    assert np.abs(Q.sum(1)).max() == 0.0
    assert Q[0, 1] == 0.8 and Q[1, 0] == 1.0


def test_request_stream():
    reqs = synth.request_stream(200)
    Ls = np.array([r["L"] for r in reqs])
    assert Ls.min() >= 128 and Ls.max() <= 16384
    assert set(r["m"] for r in reqs) <= {16, 32, 64, 128}
    assert all(0.5 <= r["ratio"] <= 0.95 for r in reqs)
    # log-uniform: median near sqrt(128*16384) = 1448
    assert 700 < np.median(Ls) < 3000
    assert reqs == synth.request_stream(200)


@pytest.mark.parametrize("p,q", [(1, 3), (2, 2), (3, 1)])
def test_banded_is_a_generator(p, q):
    L, m = 23, 5
    D = synth.banded(L, m, p, q, 0.8, seed=9)
    Q = np.zeros((L * m, L * m))
    for e, B in D.items():
        for l in range(L):
            k = l + e
            if 0 <= k < L:
                Q[l * m:(l + 1) * m, k * m:(k + 1) * m] = B[l]
            else:
                assert not B[l].any()
    off = Q - np.diag(np.diag(Q))
    assert (off >= 0).all()
    assert np.abs(Q.sum(1)).max() <= 1e-13 * np.abs(Q).max() * m
    n, _ = connected_components(sp.csr_matrix(off > 0), directed=True, connection="strong")
    assert n == 1
    l = L // 2
    up = sum(D[e][l].sum() for e in range(1, q + 1))
    dn = sum(D[e][l].sum() for e in range(-p, 0))
    assert abs(up / dn - 0.8) < 1e-13
    sub = synth.banded(L, m, p, q, 0.8, seed=9, l0=4, l1=11)
    for e in D:
        assert np.array_equal(sub[e], D[e][4:11])
