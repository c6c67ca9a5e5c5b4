"""CPU oracle for the block staircase iteration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it, and it
shares no code with the GPU library: its arithmetic lives in ``oracle.c``
(plain FP64 C, no FP contraction), wrapped here with ctypes and numpy.

What it computes (arXiv 2302.07551):
  * Eq. (1): the stationary vector pi of Q^T pi = 0, pi >= 0, e^T pi = 1;
  * Sect. 2: regular splittings T = Q^T = M - N -- stair matrices of type 1
    and 2, block Gauss-Seidel, block Jacobi -- and the normalised scheme of
    Eq. (2);
  * Algorithm 2: one staircase sweep in three steps (off-staircase products,
    diagonal-only rows, coupled rows), normalisation and the L1 step error;
  * Sect. 3: the stopping rule (step error <= eps or k >= maxit), plus the
    residual ||Q^T pi||_1 <= tol test used by the GPU solver.

Also the mixed-precision refinement step as the library defines it (not in
the paper): the operators quantized as stored (FP32, or BF16 with a
power-of-two scale per block: ``quantize_block``, ``round_bf16``), the
correction sweeps of Algorithm 2 in FP64 (``Chain.refinement_step``).

Pins (tests/test_oracle_*.py, CPU only): Example 1 and Example 2 spectra,
dense direct solves, the birth-death closed form, invariants, LU
reconstruction, equal STAIR/BGS spectra on block-tridiagonal matrices and
Young's relation with block Jacobi, observed contraction vs the eigenvalue;
BF16 rounding against hand-checked ties and torch's conversion, the FP64
refinement step against the dense correction sweeps.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

STAIR1, STAIR2, BGS, BJ = 1, 2, 3, 4
METHODS = {"stair1": STAIR1, "stair2": STAIR2, "bgs": BGS, "bj": BJ}


def build(verbose=False):
    """Compile liboracle.so in place (gcc -O2 -ffp-contract=off -fopenmp)."""
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", _SO, _SRC, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        build()
    lib = ctypes.CDLL(_SO)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.or_build_T.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp]
    lib.or_build_T.restype = None
    lib.or_lu.argtypes = [i32, vp, vp]
    lib.or_lu.restype = i32
    lib.or_lu_solve.argtypes = [i32, vp, vp, vp]
    lib.or_lu_solve.restype = None
    lib.or_factor.argtypes = [i64, i32, vp, vp, vp]
    lib.or_factor.restype = i64
    lib.or_sweep.argtypes = [i64, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.or_sweep.restype = i32
    lib.or_residual.argtypes = [i64, i32, vp, vp, vp, vp]
    lib.or_residual.restype = dbl
    lib.or_solve.argtypes = [i64, i32, i32, vp, vp, vp, vp, vp, vp, dbl, dbl, i64, i64, vp, vp]
    lib.or_solve.restype = i64
    lib.or_sweep_rhs.argtypes = [i64, i32, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.or_sweep_rhs.restype = i32
    lib.or_residual_vec.argtypes = [i64, i32, vp, vp, vp, vp, vp]
    lib.or_residual_vec.restype = None
    lib.or_sweep_banded.argtypes = [i64, i32, i32, vp, vp, vp, vp, i32, vp, vp]
    lib.or_sweep_banded.restype = i32
    lib.or_residual_banded.argtypes = [i64, i32, i32, vp, vp, vp]
    lib.or_residual_banded.restype = dbl
    lib.or_threads.argtypes = [i32]
    lib.or_threads.restype = i32
    _lib = lib
    return lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads(n=0):
    """Set (n > 0) and return the oracle's OpenMP thread count."""
    return _load().or_threads(int(n))


class Chain:
    """Blocks of T = Q^T and their LU factors for one block-tridiagonal chain.

    ``dn, loc, up`` are generator blocks of Q, shape (L, m, m), row-major:
    Q[l, l-1], Q[l, l], Q[l, l+1].
    """

    def __init__(self, dn, loc, up):
        dn, loc, up = _c64(dn), _c64(loc), _c64(up)
        L, m, m2 = loc.shape
        assert m == m2 and dn.shape == loc.shape == up.shape
        self.L, self.m, self.N = L, m, L * m
        self.Tlo = np.empty_like(loc)
        self.Tdd = np.empty_like(loc)
        self.Tup = np.empty_like(loc)
        _load().or_build_T(L, m, _p(dn), _p(loc), _p(up), _p(self.Tlo), _p(self.Tdd), _p(self.Tup))
        self.LU = np.empty_like(loc)
        self.piv = np.empty((L, m), np.int32)
        self.swaps = _load().or_factor(L, m, _p(self.Tdd), _p(self.LU), _p(self.piv))
        if self.swaps < 0:
            raise ValueError("singular diagonal block")

    def sweep(self, x, method=STAIR1):
        """Unnormalised z = M^{-1} N x for the chosen splitting."""
        x = _c64(x).reshape(-1)
        z = np.empty(self.N)
        rc = _load().or_sweep(self.L, self.m, int(method), _p(self.Tlo), _p(self.Tup),
                              _p(self.LU), _p(self.piv), _p(x), _p(z))
        if rc != 0:
            raise ValueError("bad method")
        return z

    def sweep_rhs(self, x, b, method=STAIR1):
        """z = M^{-1} (N x + b): the correction step of iterative refinement."""
        x = _c64(x).reshape(-1)
        b = _c64(b).reshape(-1)
        z = np.empty(self.N)
        rc = _load().or_sweep_rhs(self.L, self.m, int(method), _p(self.Tlo), _p(self.Tup),
                                  _p(self.LU), _p(self.piv), _p(x), _p(b), _p(z))
        if rc != 0:
            raise ValueError("bad method")
        return z

    def residual_vec(self, x):
        """r = Q^T x (the vector)."""
        x = _c64(x).reshape(-1)
        r = np.empty(self.N)
        _load().or_residual_vec(self.L, self.m, _p(self.Tlo), _p(self.Tdd), _p(self.Tup), _p(x),
                                _p(r))
        return r

    def normalised_sweep(self, x, method=STAIR1):
        """One step of Eq. (2): returns (z / e^T z, e^T z, ||z/e^T z - x||_1)."""
        x = _c64(x).reshape(-1)
        z = self.sweep(x, method)
        s = float(np.sum(z)) if self.N < 2 else float(_seqsum(z))
        pi = z / s
        return pi, s, float(np.sum(np.abs(pi - x)))

    def sweeps(self, x, k, method=STAIR1):
        """k normalised sweeps from x; returns the final iterate."""
        x = _c64(x).reshape(-1).copy()
        tmp = np.zeros(2)
        if k > 0:
            _load().or_solve(self.L, self.m, int(method), _p(self.Tlo), _p(self.Tdd), _p(self.Tup),
                             _p(self.LU), _p(self.piv), _p(x), 0.0, 0.0, int(k), 1, None, _p(tmp))
        return x

    def residual(self, x):
        """||Q^T x||_1 computed directly from the blocks."""
        x = _c64(x).reshape(-1)
        return _load().or_residual(self.L, self.m, _p(self.Tlo), _p(self.Tdd), _p(self.Tup), _p(x))

    def solve(self, x0=None, method=STAIR1, tol=1e-12, eps=0.0, maxit=100000, check_every=1,
              history=True):
        """Iterate Eq. (2) from x0 (default uniform 1/N) until resid <= tol,
        step <= eps or maxit.  Returns dict(x, sweeps, resid, step, hist)."""
        x = np.full(self.N, 1.0 / self.N) if x0 is None else _c64(x0).reshape(-1).copy()
        hist = np.zeros(maxit) if history else None
        out = np.zeros(2)
        k = _load().or_solve(self.L, self.m, int(method), _p(self.Tlo), _p(self.Tdd), _p(self.Tup),
                             _p(self.LU), _p(self.piv), _p(x), float(tol), float(eps), int(maxit),
                             int(check_every), _p(hist) if history else None, _p(out))
        if k == -1:
            raise FloatingPointError("breakdown: e^T z <= 0 or not finite")
        return dict(x=x, sweeps=int(k), resid=float(out[0]), step=float(out[1]),
                    hist=hist[:k] if history else None)

    def refinement_step(self, pi0, K, dtype="f64", apply="inverse", method=STAIR1):
        """One outer step of the mixed-precision refinement around Eq. (2), with
        the operators quantized as the library stores them and the arithmetic in
        FP64: r = Q^T pi0, q = (-T_dd)^{-1} r rounded to FP32 (dtype f32 / bf16);
        K correction sweeps from d = 0 of Algorithm 2 on Q^T d = -r, each
        diagonal-only row (then each coupled row, with the fresh neighbours)
        d_l = C_l (A_l d_{l-1} + B_l d_{l+1}) + q_l (inverse mode: A = T_lo,
        B = T_up, C = (-T_dd)^{-1} in FP32) or d_l = A_l d_{l-1} + B_l d_{l+1} + q_l
        (coupled mode: A, B = (-T_dd)^{-1} T_lo, (-T_dd)^{-1} T_up; C unused);
        then pi = (pi0 + d) / e^T (pi0 + d).  dtype f64 leaves every operator
        in FP64 (the FP64 correction step)."""
        L, m = self.L, self.m
        pi0 = _c64(pi0).reshape(-1)
        r = self.residual_vec(pi0).reshape(L, m)
        ninv = np.array([-np.linalg.solve(self.Tdd[l], np.eye(m)) for l in range(L)])
        q = np.einsum("lij,lj->li", ninv, r)
        lowp = dtype != "f64"
        if lowp:
            q = q.astype(np.float32).astype(np.float64)
        if apply == "coupled":
            A = [quantize_block(ninv[l] @ self.Tlo[l], dtype) for l in range(L)]
            B = [quantize_block(ninv[l] @ self.Tup[l], dtype) for l in range(L)]
            C = None
        else:
            A = [quantize_block(self.Tlo[l], dtype) for l in range(L)]
            B = [quantize_block(self.Tup[l], dtype) for l in range(L)]
            C = [quantize_block(ninv[l], "f32" if lowp else "f64") for l in range(L)]
        first = 0 if method == STAIR1 else 1          # parity of the diagonal-only rows
        d = np.zeros((L, m))
        for _ in range(K):
            for parity in (first, 1 - first):
                for l in range(parity, L, 2):
                    g = np.zeros(m)
                    if l > 0:
                        g += A[l] @ d[l - 1]
                    if l < L - 1:
                        g += B[l] @ d[l + 1]
                    d[l] = (g if C is None else C[l] @ g) + q[l]
        x = pi0 + d.reshape(-1)
        return x / np.sum(x)

    def iteration_matrix(self, method=STAIR1):
        """Dense M^{-1} N, column k = unnormalised sweep of e_k (small N only)."""
        assert self.N <= 4096
        G = np.empty((self.N, self.N))
        e = np.zeros(self.N)
        for k in range(self.N):
            e[:] = 0.0
            e[k] = 1.0
            G[:, k] = self.sweep(e, method)
        return G

    def dense_T(self):
        """Dense T = Q^T (small N only)."""
        L, m = self.L, self.m
        T = np.zeros((self.N, self.N))
        for l in range(L):
            T[l * m:(l + 1) * m, l * m:(l + 1) * m] = self.Tdd[l]
            if l > 0:
                T[l * m:(l + 1) * m, (l - 1) * m:l * m] = self.Tlo[l]
            if l < L - 1:
                T[l * m:(l + 1) * m, (l + 1) * m:(l + 2) * m] = self.Tup[l]
        return T


def round_bf16(x):
    """FP64 values rounded once to BF16 (8 significant bits, round to nearest,
    ties to even; zeros stay zero), returned as FP64."""
    x = np.asarray(x, np.float64)
    mant, ex = np.frexp(x)                     # x = mant 2^ex, 0.5 <= |mant| < 1
    return np.ldexp(np.rint(np.ldexp(mant, 8)), ex - 8)


def quantize_block(B, dtype):
    """A block as the mixed-precision path stores it: FP32 (round to nearest),
    or BF16 with one power-of-two scale 2^e per block, e from the block's
    largest magnitude (max |B| = f 2^e, 0.5 <= f < 1), i.e. 2^e round_bf16(B / 2^e).
    Returns the FP64 value the stored block represents."""
    B = np.asarray(B, np.float64)
    if dtype == "f32":
        return B.astype(np.float32).astype(np.float64)
    if dtype == "bf16":
        mx = np.abs(B).max()
        e = int(np.frexp(mx)[1]) if mx > 0 else 0
        return np.ldexp(round_bf16(np.ldexp(B, -e)), e)
    if dtype == "f64":
        return B.copy()
    raise ValueError(dtype)


def _seqsum(v):
    s = 0.0
    for t in v:
        s += t
    return s


def contraction(err_hist, window=50):
    """Observed contraction factor (d_k / d_{k-w})^(1/w) at the end of a run."""
    d = np.asarray(err_hist)
    w = min(window, len(d) - 1)
    return float((d[-1] / d[-1 - w]) ** (1.0 / w))


class BandedChain:
    """Block-banded T = Q^T from generator block diagonals (Algorithm 2 in full).

    diags: dict {e: array (L, m, m)} with diags[e][l] = Q[l, l+e] (row-major),
    e in [-p, q] including 0 (entries whose level l+e is outside [0, L) are
    ignored).  T blocks: T[l, l+d] = (Q[l+d, l])^T = (diags[-d][l+d])^T.
    """

    def __init__(self, diags):
        es = sorted(diags)
        L, m, _ = diags[0].shape
        self.L, self.m, self.N = L, m, L * m
        self.off = np.array(sorted(-e for e in es), dtype=np.int32)
        nd = len(self.off)
        self.TB = np.zeros((nd, L, m, m))
        for j, d in enumerate(self.off):
            G = _c64(diags[-int(d)])
            for l in range(L):
                k = l + int(d)
                if 0 <= k < L:
                    self.TB[j, l] = G[k].T
        jd = int(np.nonzero(self.off == 0)[0][0])
        self.Tdd = np.ascontiguousarray(self.TB[jd])
        self.LU = np.empty_like(self.Tdd)
        self.piv = np.empty((L, m), np.int32)
        self.swaps = _load().or_factor(L, m, _p(self.Tdd), _p(self.LU), _p(self.piv))
        if self.swaps < 0:
            raise ValueError("singular diagonal block")

    def sweep(self, x, method=STAIR1):
        x = _c64(x).reshape(-1)
        z = np.empty(self.N)
        rc = _load().or_sweep_banded(self.L, self.m, len(self.off), _p(self.off), _p(self.TB),
                                     _p(self.LU), _p(self.piv), int(method), _p(x), _p(z))
        if rc != 0:
            raise ValueError("bad method")
        return z

    def sweeps(self, x, k, method=STAIR1):
        x = _c64(x).reshape(-1).copy()
        for _ in range(k):
            z = self.sweep(x, method)
            x = z / _seqsum(z)
        return x

    def residual(self, x):
        x = _c64(x).reshape(-1)
        return _load().or_residual_banded(self.L, self.m, len(self.off), _p(self.off),
                                          _p(self.TB), _p(x))

    def solve(self, tol=1e-12, maxit=100000, check_every=1, method=STAIR1):
        x = np.full(self.N, 1.0 / self.N)
        k = 0
        r = self.residual(x)
        while k < maxit and not r <= tol:
            for _ in range(check_every):
                z = self.sweep(x, method)
                x = z / _seqsum(z)
                k += 1
            r = self.residual(x)
        return dict(x=x, sweeps=k, resid=r)

    def dense_T(self):
        L, m = self.L, self.m
        T = np.zeros((self.N, self.N))
        for j, d in enumerate(self.off):
            for l in range(L):
                k = l + int(d)
                if 0 <= k < L:
                    T[l * m:(l + 1) * m, k * m:(k + 1) * m] = self.TB[j, l]
        return T

