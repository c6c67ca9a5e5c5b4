"""GPU path vs the CPU oracle, element by element on the same seeded inputs.

Tolerances (FP64 on both sides; the only differences are summation order and
fused multiply-adds, and every product here adds terms of one sign):
  * LU factors and inverse blocks: |diff| <= 1e-13 * max|block| entrywise;
  * iterates after a fixed number K of sweeps: relative L1 <= 1e-12;
  * solutions of full solves: relative L1 <= 1e-10;
  * residuals and step errors: relative 1e-12 (absolute 1e-15 near zero).
"""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

mc = pytest.importorskip("paper_2302_07551_gb300")
nat = pytest.importorskip("paper_2302_07551_gb300._native")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l1(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).sum() / np.abs(b).sum()


def make(L, m, seed=7, dep=True, ratio=0.8):
    blocks = synth.qbd(L, m, ratio, seed, level_dependent=dep)
    return blocks, oracle.Chain(*blocks)


SHAPES = [(64, 8), (37, 5), (2, 1), (3, 33), (130, 64), (21, 100), (9, 256), (64, 1), (16, 32),
          (11, 160), (5, 113), (6, 130), (4, 200)]


@pytest.mark.parametrize("L,m", SHAPES)
def test_factor_parity(L, m):
    blocks, oc = make(L, m)
    ch = mc.Chain(*(dev(b) for b in blocks))
    LU = ch.export("lu").cpu().numpy().transpose(0, 2, 1)      # to row-major
    NI = ch.export("ninv").cpu().numpy().transpose(0, 2, 1)
    TD = ch.export("tdd").cpu().numpy().transpose(0, 2, 1)
    assert np.array_equal(TD, oc.Tdd)
    assert oc.swaps == 0
    for l in range(L):
        sc = np.abs(oc.LU[l]).max()
        assert np.abs(LU[l] - oc.LU[l]).max() <= 1e-13 * sc, l
        ref = -np.linalg.inv(oc.Tdd[l])
        assert np.abs(NI[l] - ref).max() <= 1e-13 * np.abs(ref).max(), l
        assert (NI[l] >= 0).all()
    ch.close()


@pytest.mark.parametrize("apply", ["inverse", "coupled"])
@pytest.mark.parametrize("stair", [1, 2])
@pytest.mark.parametrize("L,m", SHAPES)
def test_iterates_after_fixed_sweeps(L, m, stair, apply):
    K = 50
    blocks, oc = make(L, m, seed=L * 31 + m)
    ch = mc.Chain(*(dev(b) for b in blocks), stair=stair, apply=apply)
    N = L * m
    x0 = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    stats = torch.zeros(3, dtype=torch.float64, device="cuda")
    x = ch.sweep(x0, nsweeps=K, stats=stats)
    ref = oc.sweeps(np.full(N, 1.0 / N), K, method=oracle.STAIR1 if stair == 1 else oracle.STAIR2)
    assert rel_l1(x.cpu().numpy(), ref) <= 1e-12
    # step error and e^T z of the last sweep
    prev = oc.sweeps(np.full(N, 1.0 / N), K - 1, method=oracle.STAIR1 if stair == 1 else oracle.STAIR2)
    pi, s, d = oc.normalised_sweep(prev, oracle.STAIR1 if stair == 1 else oracle.STAIR2)
    st = stats.cpu().numpy()
    assert abs(st[0] - s) <= 1e-12 * abs(s)
    # the step error is a difference of two unit-L1 vectors: absolute bound,
    # consistent with the 1e-12 relative L1 bound on the iterates
    assert abs(st[1] - d) <= 1e-12
    ch.close()


U = 2.0 ** -53


def abs_bound(oc, x):
    """|| |Q^T| |x| ||_1: the scale of the rounding error of any FP64
    evaluation of Q^T x (every term of every row summed in absolute value)."""
    L, m = oc.L, oc.m
    P = np.abs(np.asarray(x, np.float64)).reshape(L, m)
    B = 0.0
    for l in range(L):
        acc = np.abs(oc.Tdd[l]) @ P[l]
        if l > 0:
            acc += np.abs(oc.Tlo[l]) @ P[l - 1]
        if l < L - 1:
            acc += np.abs(oc.Tup[l]) @ P[l + 1]
        B += acc.sum()
    return B


def resid_tol(oc, x, r):
    """Allowed |r_gpu - r_oracle| for ||Q^T x||_1: both sides are exact up to
    rounding of sums of at most 3m products (plus, on the GPU, the rounding of
    the sweep that produced x), each bounded by a small multiple of m u B."""
    return 1e-12 * r + 8 * oc.m * U * abs_bound(oc, x)


@pytest.mark.parametrize("apply", ["inverse", "coupled"])
@pytest.mark.parametrize("stair", [1, 2])
@pytest.mark.parametrize("L,m", [(64, 8), (37, 5), (2, 1), (3, 33), (130, 64), (21, 100),
                                 (9, 256), (11, 160)])
def test_sweep_residual_from_the_splitting(L, m, stair, apply):
    """stats[2] of a sweep call is ||Q^T pi||_1 of the returned pi, formed from
    the splitting (Q^T z = N (x - z), zero on the coupled rows) at the end of
    the fused launch; it matches the oracle's direct residual of the same pi
    within the rounding bound (sharp while the residual is far above it)."""
    blocks, oc = make(L, m, seed=L * 17 + m)
    ch = mc.Chain(*(dev(b) for b in blocks), stair=stair, apply=apply)
    N = L * m
    x0 = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    for K in (1, 2, 7, 50):
        st = torch.zeros(3, dtype=torch.float64, device="cuda")
        x = ch.sweep(x0, nsweeps=K, stats=st).cpu().numpy()
        r_gpu = float(st[2])
        r_or = oc.residual(x)
        tol = resid_tol(oc, x, r_or)
        assert abs(r_gpu - r_or) <= tol, (K, r_gpu, r_or, tol)
        if r_or > 1e3 * tol:       # far from the rounding floor: a sharp check
            assert abs(r_gpu - r_or) <= 1e-6 * r_or
    ch.sync()
    ch.close()


@pytest.mark.parametrize("Lp,mp", [(12, 32), (8, 128)])
def test_paired_sweep_residual_from_the_splitting(Lp, mp):
    """Paired pentadiagonal chains: the residual products skip the zero
    quadrants of T_lo / T_up, as the sweep does."""
    blocks = synth.penta_paired(Lp, mp, 0.8, 0.3, seed=Lp * mp)
    oc = oracle.Chain(*blocks)
    ch = mc.Chain(*(dev(b) for b in blocks), paired=True)
    N = Lp * mp
    x0 = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    for K in (1, 9):
        st = torch.zeros(3, dtype=torch.float64, device="cuda")
        x = ch.sweep(x0, nsweeps=K, stats=st).cpu().numpy()
        r_or = oc.residual(x)
        assert abs(float(st[2]) - r_or) <= resid_tol(oc, x, r_or)
        assert abs(float(st[2]) - r_or) <= 1e-6 * r_or
    ch.sync()
    ch.close()


def test_solve_stops_at_the_oracles_sweep_with_per_sweep_checks():
    """check_every = 1: the solve tests the residual (from the splitting,
    confirmed by the direct residual) after every sweep and stops at the
    oracle's first sweep with ||Q^T pi||_1 <= tol (unless that residual lies
    within rounding of tol, where either neighbouring sweep is correct)."""
    blocks = synth.workload("qbd_L64_m8")
    oc = oracle.Chain(*blocks)
    tol = 1e-12
    ref = oc.solve(tol=tol, maxit=100000, check_every=1)
    k = ref["sweeps"]
    N = oc.N
    r_k = ref["resid"]
    x_prev = oc.sweeps(np.full(N, 1.0 / N), k - 1)
    r_prev = oc.residual(x_prev)
    ch = mc.Chain(*(dev(b) for b in blocks))
    pi, res = ch.solve(tol=tol, maxit=100000, check_every=1)
    ch.close()
    band = resid_tol(oc, ref["x"], tol)
    if abs(r_k - tol) > band and abs(r_prev - tol) > band:
        assert res["sweeps"] == k
    else:
        assert abs(res["sweeps"] - k) <= 1
    assert res["converged"] and res["residual"] <= tol
    assert rel_l1(pi.cpu().numpy(), ref["x"]) <= 1e-10


def test_banded_sweep_stats_carry_the_direct_residual():
    """Block-banded chains (off-staircase terms on every row) report the
    direct residual of the result in stats[2]."""
    D = synth.banded(20, 16, 1, 3, 0.8, seed=3)
    bc = oracle.BandedChain(D)
    ch = mc.Chain.banded({e: dev(B) for e, B in D.items()})
    N = 20 * 16
    st = torch.zeros(3, dtype=torch.float64, device="cuda")
    x = ch.sweep(torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda"), nsweeps=5,
                 stats=st).cpu().numpy()
    r = bc.residual(x)
    assert abs(float(st[2]) - r) <= 1e-12 * r
    ch.sync()
    ch.close()


def test_one_sweep_from_random_vector():
    L, m = 33, 48
    blocks, oc = make(L, m, seed=3)
    ch = mc.Chain(*(dev(b) for b in blocks))
    x = np.random.default_rng(1).random(L * m)
    x /= x.sum()
    out = ch.sweep(dev(x)).cpu().numpy()
    ref, _, _ = oc.normalised_sweep(x)
    assert rel_l1(out, ref) <= 1e-13
    ch.close()


@pytest.mark.parametrize("stair,apply", [(1, "inverse"), (2, "coupled")])
def test_gpu_sweep_zeroes_the_coupled_rows_of_the_residual(stair, apply):
    """Property of the stair splitting (M z = N x row by row, N = 0 on the
    coupled rows): the GPU iterate after a sweep has Q^T pi = 0 on every
    coupled block row, to rounding, at a size that spans many warps."""
    L, m = 200, 48
    blocks, oc = make(L, m, seed=33)
    ch = mc.Chain(*(dev(b) for b in blocks), stair=stair, apply=apply)
    x = np.random.default_rng(8).random(L * m)
    x /= x.sum()
    for n in (1, 3):
        pi = ch.sweep(dev(x), nsweeps=n).cpu().numpy()
        r = oc.residual_vec(pi).reshape(L, m)
        coupled = np.arange(L) % 2 == (1 if stair == 1 else 0)
        assert np.abs(r[coupled]).sum() <= 1e-13 * np.abs(r).sum() + 1e-18, n
        assert np.abs(r[~coupled]).sum() > 0
    ch.sync()
    ch.close()


def test_residual_parity():
    for (L, m) in [(64, 8), (19, 70), (5, 256)]:
        blocks, oc = make(L, m, seed=L)
        ch = mc.Chain(*(dev(b) for b in blocks))
        x = np.random.default_rng(L).random(L * m)
        r = ch.residual(dev(x))
        ref = oc.residual(x)
        assert abs(r - ref) <= 1e-12 * ref
        ch.close()


def test_solution_parity_qbd_L64_m8():
    blocks = synth.workload("qbd_L64_m8")
    oc = oracle.Chain(*blocks)
    ref = oc.solve(tol=1e-12, maxit=100000, check_every=32)
    ch = mc.Chain(*(dev(b) for b in blocks))
    pi, res = ch.solve(tol=1e-12, maxit=100000, check_every=32)
    assert res["converged"] and res["residual"] <= 1e-12
    assert res["sweeps"] == ref["sweeps"]
    pi = pi.cpu().numpy()
    assert rel_l1(pi, ref["x"]) <= 1e-10
    assert (pi >= 0).all() and abs(pi.sum() - 1) <= 1e-13
    assert 0.97 < res["contraction"] < 1.0
    ch.close()


def test_birth_death_closed_form_on_gpu():
    L, lam, mu = 64, 0.8, 1.0
    blocks = synth.birth_death(L, lam, mu)
    ch = mc.Chain(*(dev(b) for b in blocks))
    pi, res = ch.solve(tol=1e-15, maxit=200000, check_every=64)
    r = lam / mu
    ref = (1 - r) * r ** np.arange(L) / (1 - r ** L)
    assert rel_l1(pi.cpu().numpy(), ref) <= 1e-11
    ch.close()


def test_deterministic_and_checkpoint_resume():
    """Equal calls are bitwise equal (units are claimed dynamically, but every
    value and every sum is fixed by the level order); resuming from a stored
    iterate agrees up to rounding (the sweeps of one call are not normalised
    in between, Eq. (2) is scale-invariant)."""
    L, m = 300, 64
    blocks, _ = make(L, m, seed=5)
    ch = mc.Chain(*(dev(b) for b in blocks))
    N = L * m
    x0 = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    st_a = torch.zeros(3, dtype=torch.float64, device="cuda")
    st_b = torch.zeros(3, dtype=torch.float64, device="cuda")
    a = ch.sweep(x0, nsweeps=20, stats=st_a)
    for _ in range(3):
        b = ch.sweep(x0, nsweeps=20, stats=st_b)
        assert torch.equal(a, b) and torch.equal(st_a[:2], st_b[:2])
    half = ch.sweep(x0, nsweeps=10).clone()          # checkpoint = the pi tensor
    c = ch.sweep(half, nsweeps=10)
    assert rel_l1(a.cpu().numpy(), c.cpu().numpy()) <= 1e-14
    ch.sync()
    ch.close()


def test_solve_from_x0_and_stair2_agree():
    blocks, oc = make(40, 12, seed=9)
    ref = oc.solve(tol=1e-13, maxit=100000, check_every=16)["x"]
    N = 40 * 12
    x0 = torch.rand(N, dtype=torch.float64, device="cuda")
    for stair in (1, 2):
        for apply in ("inverse", "coupled"):
            ch = mc.Chain(*(dev(b) for b in blocks), stair=stair, apply=apply)
            pi, res = ch.solve(x0=x0, tol=1e-13, maxit=100000, check_every=16)
            assert rel_l1(pi.cpu().numpy(), ref) <= 1e-10
            ch.close()


# --- error behaviour (no fault, no hang) ---------------------------------------------

def test_errors_reported():
    blocks, _ = make(8, 4, seed=2)
    d = [dev(b) for b in blocks]
    ch = mc.Chain(*d, factor=False)
    x = torch.full((32,), 1 / 32, dtype=torch.float64, device="cuda")
    with pytest.raises(mc.McError) as e:
        ch.sweep(x)
    assert e.value.status == 5                       # not factored
    ch.factor()
    with pytest.raises(mc.McError) as e:
        ch.solve(x0=-x)
    assert e.value.status == 1                       # x0 negative
    pi, res = ch.solve(tol=1e-300, maxit=5, raise_on_maxit=False)
    assert res["status"] == 7 and res["sweeps"] == 5
    ch.close()
    # a level with no rates at all: zero diagonal block
    loc = d[1].clone()
    loc[3] = 0.0
    with pytest.raises(mc.McError) as e:
        mc.Chain(d[0], loc, d[2])
    assert e.value.status == 4
    # non-finite rate off the diagonal blocks: normalisation breaks down
    up = d[2].clone()
    up[2, 0, 1] = float("nan")
    ch = mc.Chain(d[0], d[1], up)
    with pytest.raises(mc.McError) as e:
        ch.solve(tol=1e-12, maxit=64, check_every=8)
    assert e.value.status == 6
    # the latch was cleared: the next call runs without raising (its value is
    # NaN, the blocks hold a NaN)
    ch.residual(x)
    ch.close()


# --- full size, launch configuration of the benchmark --------------------------------

@pytest.mark.slow
def test_full_size_qbd_L32768_m64_sampled():
    """L=32768, m=64: GPU sweep k+1 against the oracle's sweep of the GPU
    iterate k on sampled level windows (the sweep is local: rows of a window
    depend only on the window and its neighbours)."""
    name = "qbd_L32768_m64"
    w = synth.WORKLOADS[name]
    L, m = w["L"], w["m"]
    blocks = synth.workload(name)
    ch = mc.Chain(*(dev(b) for b in blocks))
    del blocks
    N = L * m
    x = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    xk = ch.sweep(x, nsweeps=7)
    stats = torch.zeros(3, dtype=torch.float64, device="cuda")
    xk1 = ch.sweep(xk, nsweeps=1, stats=stats)
    s = float(stats[0])
    xk = xk.cpu().numpy()
    xk1 = xk1.cpu().numpy()
    for a in (0, 2, 10000, 32768 - 40):
        b = min(a + 40, L)
        wb = synth.qbd(L, m, w["ratio"], w["seed"], True, a, b)
        sub = oracle.Chain(*wb)
        z = sub.sweep(xk[a * m:b * m])
        lo = a if a == 0 else a + 2
        hi = b if b == L else b - 2
        got = xk1[lo * m:hi * m]
        ref = z[(lo - a) * m:(hi - a) * m] / s
        assert rel_l1(got, ref) <= 1e-12, a
    # and e^T x = 1, x >= 0 at full size
    assert abs(xk1.sum() - 1) <= 1e-12 and (xk1 >= 0).all()
    ch.close()


@pytest.mark.slow
@pytest.mark.parametrize("name", ["qbd_L16384_m256", "penta_L8192_m128"])
def test_full_size_sampled_other_workloads(name):
    """The other FP64 bench workloads at full size, in the bench's launch
    configuration (fused sweeps; the pentadiagonal chain paired into 4096
    super-levels of 256 with the zero quadrants skipped): GPU sweep k+1
    against the oracle's sweep of the GPU iterate k on sampled windows."""
    L, m = synth.workload_shape(name)
    paired = synth.WORKLOADS[name]["kind"] == "penta"
    blocks = synth.workload(name)
    ch = mc.Chain(*(dev(b) for b in blocks), paired=paired)
    del blocks
    N = L * m
    x = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    xk = ch.sweep(x, nsweeps=4)
    stats = torch.zeros(3, dtype=torch.float64, device="cuda")
    xk1 = ch.sweep(xk, nsweeps=1, stats=stats)
    s = float(stats[0])
    xk = xk.cpu().numpy()
    xk1 = xk1.cpu().numpy()
    for a in (0, 2, L // 2, L - 24):     # even starts: the window keeps the global parity
        b = min(a + 24, L)
        sub = oracle.Chain(*synth.workload(name, a, b))
        z = sub.sweep(xk[a * m:b * m])
        lo = a if a == 0 else a + 2
        hi = b if b == L else b - 2
        got = xk1[lo * m:hi * m]
        ref = z[(lo - a) * m:(hi - a) * m] / s
        assert rel_l1(got, ref) <= 1e-12, (name, a)
    assert abs(xk1.sum() - 1) <= 1e-12 and (xk1 >= 0).all()
    ch.sync()
    ch.close()


# --- paired block-pentadiagonal chains: zero quadrants skipped ------------------------

@pytest.mark.parametrize("Lp,mp", [(12, 32), (10, 64), (8, 128), (9, 96)])
def test_paired_pentadiagonal_skips_zero_quadrants(Lp, mp):
    """Levels of a chain with jumps of +-1, +-2 paired into blocks of 2 mp:
    the sweep that skips the structurally zero quadrants equals the oracle's
    dense sweep, as does the residual."""
    if Lp % 2:
        Lp += 1
    blocks = synth.penta_paired(Lp, mp, 0.8, 0.3, seed=Lp + mp)
    oc = oracle.Chain(*blocks)
    L, m = Lp // 2, 2 * mp
    if m % 64:
        with pytest.raises(ValueError):
            mc.Chain(*(dev(b) for b in blocks), paired=True)
        return
    ch = mc.Chain(*(dev(b) for b in blocks), paired=True)
    N = L * m
    x0 = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    x = ch.sweep(x0, nsweeps=30).cpu().numpy()
    ref = oc.sweeps(np.full(N, 1.0 / N), 30)
    assert rel_l1(x, ref) <= 1e-12
    y = np.random.default_rng(1).random(N)
    assert abs(ch.residual(dev(y)) - oc.residual(y)) <= 1e-12 * oc.residual(y)
    pi, res = ch.solve(tol=1e-12, maxit=200000, check_every=32)
    sol = oc.solve(tol=1e-13, maxit=200000, check_every=32)["x"]
    assert rel_l1(pi.cpu().numpy(), sol) <= 1e-10
    ch.close()


def test_paired_chain_in_coupled_mode():
    """A paired pentadiagonal chain in coupled mode (dense W blocks: the
    products no longer have zero quadrants, so nothing is skipped) and in
    STAIR2 order: iterates and solution as the oracle's."""
    blocks = synth.penta_paired(20, 64, 0.8, 0.3, seed=31)
    oc = oracle.Chain(*blocks)
    L, m = 10, 128
    N = L * m
    for stair, meth in ((1, oracle.STAIR1), (2, oracle.STAIR2)):
        ch = mc.Chain(*(dev(b) for b in blocks), paired=True, apply="coupled", stair=stair)
        x = ch.sweep(torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda"), nsweeps=25)
        assert rel_l1(x.cpu().numpy(), oc.sweeps(np.full(N, 1.0 / N), 25, method=meth)) <= 1e-12
        pi, res = ch.solve(tol=1e-12, maxit=200000, check_every=32)
        sol = oc.solve(tol=1e-13, maxit=200000, check_every=32)["x"]
        assert res["converged"] and rel_l1(pi.cpu().numpy(), sol) <= 1e-10
        ch.close()


def test_paired_flag_rejects_dense_off_diagonal_blocks():
    blocks = synth.qbd(6, 64, 0.8, seed=3)
    with pytest.raises(mc.McError) as e:
        mc.Chain(*(dev(b) for b in blocks), paired=True)
    assert e.value.status == 1


# --- comparison splittings of Sect. 2 on the GPU --------------------------------------

@pytest.mark.parametrize("stair,meth", [(3, oracle.BJ), (4, oracle.BGS)])
@pytest.mark.parametrize("L,m", [(37, 5), (64, 64), (9, 160)])
def test_block_jacobi_and_gauss_seidel_sweeps(stair, meth, L, m):
    K = 20
    blocks, oc = make(L, m, seed=L + 7 * m)
    ch = mc.Chain(*(dev(b) for b in blocks), stair=stair)
    N = L * m
    x = ch.sweep(torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda"), nsweeps=K)
    ref = oc.sweeps(np.full(N, 1.0 / N), K, method=meth)
    assert rel_l1(x.cpu().numpy(), ref) <= 1e-12
    ch.close()


@pytest.mark.parametrize("apply", ["inverse", "coupled"])
@pytest.mark.parametrize("L,m", [(64, 8), (37, 5), (2, 1), (3, 33), (130, 64), (9, 256),
                                 (11, 160), (300, 16)])
def test_fused_block_gauss_seidel_sweeps(L, m, apply):
    """Block Gauss-Seidel sweeps in one wavefront-ordered fused launch: the
    iterates, e^T z, the step error and the (direct) residual of the last
    sweep as the oracle's, out of place and in place."""
    blocks, oc = make(L, m, seed=L * 5 + m)
    ch = mc.Chain(*(dev(b) for b in blocks), stair=4, apply=apply)
    N = L * m
    x0 = np.random.default_rng(L + m).random(N)
    x0 /= x0.sum()
    for K in (1, 2, 50):
        prev = oc.sweeps(x0, K - 1, method=oracle.BGS) if K > 1 else x0
        ref, s, d = oc.normalised_sweep(prev, oracle.BGS)
        for in_place in (False, True):
            x = dev(x0.copy())
            st = torch.zeros(3, dtype=torch.float64, device="cuda")
            out = ch.sweep(x, x if in_place else None, nsweeps=K, stats=st).cpu().numpy()
            assert rel_l1(out, ref) <= 1e-12, (K, in_place)
            g = st.cpu().numpy()
            assert abs(g[0] - s) <= 1e-12 * abs(s) and abs(g[1] - d) <= 1e-12
            r = oc.residual(out)
            assert abs(g[2] - r) <= resid_tol(oc, out, r)
    ch.sync()
    ch.close()


def test_fused_block_gauss_seidel_beyond_one_launch():
    """More block Gauss-Seidel sweeps than one fused launch takes (1024)."""
    L, m, K = 24, 8, 1100
    blocks, oc = make(L, m, seed=23)
    ch = mc.Chain(*(dev(b) for b in blocks), stair=4)
    N = L * m
    x = ch.sweep(torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda"), nsweeps=K)
    ref = oc.sweeps(np.full(N, 1.0 / N), K, method=oracle.BGS)
    assert rel_l1(x.cpu().numpy(), ref) <= 1e-12
    ch.sync()
    ch.close()


def test_contraction_stair_equals_gauss_seidel_and_jacobi_stalls():
    """Sect. 2: on block-tridiagonal Q^T the staircase iteration converges at
    the block Gauss-Seidel rate; block Jacobi has |lambda| = 1 twice."""
    blocks = synth.workload("qbd_L64_m8")
    kap = {}
    for stair in (1, 2, 4):
        ch = mc.Chain(*(dev(b) for b in blocks), stair=stair)
        _, res = ch.solve(tol=0.0, eps=1e-13, maxit=20000, check_every=100)
        kap[stair] = res["contraction"]
        ch.close()
    assert abs(kap[1] - kap[4]) < 2e-3 and abs(kap[2] - kap[4]) < 2e-3
    gamma = sorted(abs(np.linalg.eigvals(oracle.Chain(*blocks).iteration_matrix(oracle.BGS))))[-2]
    assert abs(kap[1] - gamma) < 2e-3
    ch = mc.Chain(*(dev(b) for b in blocks), stair=3)
    _, res = ch.solve(tol=0.0, eps=1e-13, maxit=2000, check_every=100, raise_on_maxit=False)
    assert res["status"] == 7 and res["step"] > 1e-6     # block Jacobi does not converge
    ch.close()


@pytest.mark.parametrize("stair,apply", [(1, "inverse"), (2, "coupled")])
def test_multi_sweep_call_equals_single_sweeps(stair, apply):
    """n sweeps in one fused launch (no normalisation in between) equal n
    normalised single sweeps up to rounding, including e^T z of the last sweep
    relative to the previous iterate and the step error."""
    blocks, _ = make(45, 24, seed=8)
    ch = mc.Chain(*(dev(b) for b in blocks), stair=stair, apply=apply)
    N = 45 * 24
    x0 = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    for n in (2, 3, 7, 40):
        st_a = torch.zeros(3, dtype=torch.float64, device="cuda")
        st_b = torch.zeros(3, dtype=torch.float64, device="cuda")
        a = ch.sweep(x0, nsweeps=n, stats=st_a)
        b = x0.clone()
        for _ in range(n):
            b = ch.sweep(b, nsweeps=1, stats=st_b)
        assert rel_l1(a.cpu().numpy(), b.cpu().numpy()) <= 1e-14
        sa, sb = st_a.cpu().numpy(), st_b.cpu().numpy()
        assert abs(sa[0] - sb[0]) <= 1e-14 * abs(sb[0])
        assert abs(sa[1] - sb[1]) <= 1e-14
    ch.sync()
    ch.close()


def test_sweeps_beyond_one_fused_launch():
    """More sweeps than one fused launch takes (1024): the launches chain with
    a normalisation in between; iterates and stats as the oracle's."""
    L, m, K = 24, 8, 1100
    blocks, oc = make(L, m, seed=21)
    ch = mc.Chain(*(dev(b) for b in blocks))
    N = L * m
    x0 = np.random.default_rng(2).random(N)
    x0 /= x0.sum()
    stats = torch.zeros(3, dtype=torch.float64, device="cuda")
    x = ch.sweep(dev(x0), nsweeps=K, stats=stats)
    prev = oc.sweeps(x0, K - 1)
    ref, s, d = oc.normalised_sweep(prev)
    assert rel_l1(x.cpu().numpy(), ref) <= 1e-12
    st = stats.cpu().numpy()
    assert abs(st[0] - s) <= 1e-12 * abs(s) and abs(st[1] - d) <= 1e-12
    r = oc.residual(x.cpu().numpy())
    assert abs(st[2] - r) <= resid_tol(oc, x.cpu().numpy(), r)
    ch.sync()
    ch.close()


def test_in_place_single_and_multi_sweep():
    """x_in == x_out: the first half-sweep reads x_in while the second writes
    it (only after both readers of a level are done); the step error of a
    single in-place sweep still sees the old iterate."""
    L, m = 37, 40
    blocks, oc = make(L, m, seed=4)
    ch = mc.Chain(*(dev(b) for b in blocks))
    N = L * m
    x0 = np.random.default_rng(5).random(N)
    x0 /= x0.sum()
    for n in (1, 5):
        x = dev(x0.copy())
        stats = torch.zeros(3, dtype=torch.float64, device="cuda")
        ch.sweep(x, x, nsweeps=n, stats=stats)
        prev = oc.sweeps(x0, n - 1) if n > 1 else x0
        ref, s, d = oc.normalised_sweep(prev)
        assert rel_l1(x.cpu().numpy(), ref) <= 1e-13
        assert abs(float(stats[1]) - d) <= 1e-13
    ch.sync()
    ch.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_sweeps_equal_device_sweeps(pinned):
    """mc_sweep_host (pinned output: the normalisation writes it directly;
    pageable: copied back) gives bitwise the device call's iterate and stats,
    in place and out of place."""
    L, m = 37, 24
    blocks, _ = make(L, m, seed=12)
    ch = mc.Chain(*(dev(b) for b in blocks))
    N = L * m
    x0 = torch.rand(N, dtype=torch.float64)
    x0 /= x0.sum()
    for n in (1, 4):
        st = torch.zeros(3, dtype=torch.float64, device="cuda")
        ref = ch.sweep(x0.cuda(), nsweeps=n, stats=st).cpu()
        xh = x0.clone().pin_memory() if pinned else x0.clone()
        yh = torch.empty(N, dtype=torch.float64)
        yh = yh.pin_memory() if pinned else yh
        sh = ch.sweep_host(xh, yh, n)
        assert torch.equal(yh, ref) and sh[0] == float(st[0]) and sh[1] == float(st[1])
        assert sh[2] == float(st[2])
        zh = torch.empty(N, dtype=torch.float64)
        zh = zh.pin_memory() if pinned else zh
        assert ch.sweep_host(xh, zh, n, stats=False) is None     # no residual formed
        assert torch.equal(zh, ref)
        sh = ch.sweep_host(xh, xh, n)                     # in place
        assert torch.equal(xh, ref)
    ch.sync()
    ch.close()


def test_bounded_wait_reports_instead_of_hanging():
    """The wait between units of a fused launch gives up after its limit and
    latches MC_ERR_TIMEOUT; a satisfiable wait returns at once."""
    lib = nat.load()
    s = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    assert lib.mc_wait_selftest(ctypes.c_void_p(s), 0, 20_000_000) == nat.MC_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert lib.mc_wait_selftest(ctypes.c_void_p(s), 1, 20_000_000) == 0
    # the context stays usable
    blocks, oc = make(8, 4)
    ch = mc.Chain(*(dev(b) for b in blocks))
    ch.sweep(torch.full((32,), 1 / 32, dtype=torch.float64, device="cuda"), nsweeps=3)
    ch.sync()
    ch.close()


# --- block-banded chains: Algorithm 2 with off-staircase terms ------------------------

@pytest.mark.parametrize("L,m,p,q", [(40, 16, 1, 4), (33, 64, 3, 1), (21, 40, 2, 3), (12, 160, 1, 2)])
def test_banded_sweeps_residual_and_solve(L, m, p, q):
    D = synth.banded(L, m, p, q, 0.8, seed=L + m + p)
    bc = oracle.BandedChain(D)
    dd = {e: dev(B) for e, B in D.items()}
    N = L * m
    for stair, meth in ((1, oracle.STAIR1), (2, oracle.STAIR2), (3, oracle.BJ), (4, oracle.BGS)):
        ch = mc.Chain.banded(dd, stair=stair)
        x = ch.sweep(torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda"), nsweeps=15)
        ref = bc.sweeps(np.full(N, 1.0 / N), 15, method=meth)
        assert rel_l1(x.cpu().numpy(), ref) <= 1e-12, stair
        ch.close()
    ch = mc.Chain.banded(dd)
    y = np.random.default_rng(2).random(N)
    assert abs(ch.residual(dev(y)) - bc.residual(y)) <= 1e-12 * bc.residual(y)
    pi, res = ch.solve(tol=1e-12, maxit=200000, check_every=32)
    sol = bc.solve(tol=1e-13, maxit=200000, check_every=50)["x"]
    assert res["converged"] and rel_l1(pi.cpu().numpy(), sol) <= 1e-10
    ch.close()


@pytest.mark.parametrize("stair", [1, 2])
def test_banded_fused_stats_and_in_place(stair):
    """Block-banded fused launches alternate two buffers: e^T z of the last
    sweep (relative to the previous iterate) and the step error after K = 1,
    2, 3 and 9 sweeps, in place and out of place, as the oracle's."""
    L, m, p, q = 26, 24, 2, 4
    D = synth.banded(L, m, p, q, 0.8, seed=7)
    bc = oracle.BandedChain(D)
    meth = oracle.STAIR1 if stair == 1 else oracle.STAIR2
    ch = mc.Chain.banded({e: dev(B) for e, B in D.items()}, stair=stair)
    N = L * m
    x0 = np.random.default_rng(9).random(N)
    x0 /= x0.sum()
    for K in (1, 2, 3, 9):
        prev = bc.sweeps(x0, K - 1, method=meth) if K > 1 else x0
        z = bc.sweep(prev, method=meth)
        ref = z / z.sum()
        for in_place in (False, True):
            x = dev(x0.copy())
            st = torch.zeros(3, dtype=torch.float64, device="cuda")
            out = ch.sweep(x, x if in_place else None, nsweeps=K, stats=st)
            assert rel_l1(out.cpu().numpy(), ref) <= 1e-12, (K, in_place)
            s, d = st.cpu().numpy()[:2]
            assert abs(s - z.sum()) <= 1e-12 * abs(z.sum())
            assert abs(d - np.abs(ref - prev).sum()) <= 1e-12
    ch.sync()
    ch.close()


def test_banded_sweeps_beyond_one_fused_launch():
    """Block-banded chain, more sweeps than one fused launch takes: the
    launches chain through a normalisation and restart their alternating
    buffers; iterates and stats as the oracle's."""
    L, m, p, q, K = 14, 8, 1, 3, 1030
    D = synth.banded(L, m, p, q, 0.8, seed=17)
    bc = oracle.BandedChain(D)
    ch = mc.Chain.banded({e: dev(B) for e, B in D.items()})
    N = L * m
    x0 = np.random.default_rng(4).random(N)
    x0 /= x0.sum()
    st = torch.zeros(3, dtype=torch.float64, device="cuda")
    x = ch.sweep(dev(x0), nsweeps=K, stats=st)
    prev = bc.sweeps(x0, K - 1)
    z = bc.sweep(prev)
    ref = z / z.sum()
    assert rel_l1(x.cpu().numpy(), ref) <= 1e-12
    s, d = st.cpu().numpy()[:2]
    assert abs(s - z.sum()) <= 1e-12 * abs(z.sum()) and abs(d - np.abs(ref - prev).sum()) <= 1e-12
    ch.sync()
    ch.close()


def test_banded_restrictions():
    D = {e: dev(B) for e, B in synth.banded(8, 8, 1, 3, 0.8, seed=1).items()}
    for kw in (dict(apply="coupled"), dict(dtype="f32")):
        with pytest.raises(ValueError):
            mc.Chain.banded(D, **kw)


def test_banded_host_buffer_sweeps_and_tuning():
    """Block-banded chain: mc_sweep_host with stats (the direct residual of the
    result) equals the device call bitwise; mc_tune on banded and block
    Gauss-Seidel chains keeps a configuration that changes no iterate."""
    D = synth.banded(30, 16, 1, 3, 0.8, seed=11)
    bc = oracle.BandedChain(D)
    ch = mc.Chain.banded({e: dev(B) for e, B in D.items()})
    N = 30 * 16
    x0 = torch.rand(N, dtype=torch.float64)
    x0 /= x0.sum()
    st = torch.zeros(3, dtype=torch.float64, device="cuda")
    ref = ch.sweep(x0.cuda(), nsweeps=4, stats=st).cpu()
    xh = x0.clone().pin_memory()
    yh = torch.empty(N, dtype=torch.float64).pin_memory()
    sh = ch.sweep_host(xh, yh, 4)
    assert torch.equal(yh, ref) and sh[2] == float(st[2])
    assert abs(sh[2] - bc.residual(ref.numpy())) <= 1e-12 * bc.residual(ref.numpy())
    for chain in (ch, mc.Chain(*(dev(b) for b in synth.qbd(40, 24, 0.8, seed=3)), stair=4)):
        x = torch.full((chain.N,), 1.0 / chain.N, dtype=torch.float64, device="cuda")
        a = chain.sweep(x, nsweeps=9).clone()
        bps, lpu, ms = chain.tune(x, 9)
        assert lpu == 1 and ms > 0
        for b in (0, 1, 2):
            chain.set_tuning(b, 1)
            assert torch.equal(chain.sweep(x, nsweeps=9), a)
        chain.sync()
        chain.close()
