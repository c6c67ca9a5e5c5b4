"""Seeded synthetic Markov-generator inputs (problem data only, no solver arithmetic).

Every block is produced by ``synth.c`` from a counter-based SplitMix64 hash, so
a given (seed, sizes) always yields bit-identical FP64 blocks on any machine,
for any thread count and for any subrange of levels.  The CPU oracle and the
GPU library both take their inputs from here; neither imports the other.

Blocks are generator blocks of Q, row-major ``[levels][m][m]`` float64:
``dn[l] = Q[l, l-1]``, ``loc[l] = Q[l, l]``, ``up[l] = Q[l, l+1]``
(``dn[0]`` and ``up[L-1]`` are zero).  The transposed system ``Q^T pi = 0``
of Eq. (1) is what the solvers work on.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None

# Workloads, named by what they are.  Seeds equal the workload index 0..4.
WORKLOADS = {
    # L=64, m=8, level-independent, up/down ratio 0.8
    "qbd_L64_m8": dict(kind="qbd", L=64, m=8, ratio=0.8, level_dependent=False, seed=0),
    # m=1 birth-death chain, lambda=0.8, mu=1 (closed form (1-r) r^i / (1-r^L))
    "birth_death_L64": dict(kind="birth_death", L=64, m=1, lam=0.8, mu=1.0),
    # L=32768, m=64, level-dependent, ratio 0.9 (FP64 blocks ~3.2 GB)
    "qbd_L32768_m64": dict(kind="qbd", L=32768, m=64, ratio=0.9, level_dependent=True, seed=1),
    # same recipe at L=512: contraction comparisons that run to the asymptotic regime
    "qbd_L512_m64": dict(kind="qbd", L=512, m=64, ratio=0.9, level_dependent=True, seed=1),
    # same recipe at L=8192 (0.8 GB of blocks per sweep): profiling-size case
    "qbd_L8192_m64": dict(kind="qbd", L=8192, m=64, ratio=0.9, level_dependent=True, seed=1),
    # same recipe at L=2048 (L/16 of the bench chain): solution parity with the oracle
    "qbd_L2048_m64": dict(kind="qbd", L=2048, m=64, ratio=0.9, level_dependent=True, seed=1),
    # block Hessenberg: batch arrivals of up to 4 levels, single-level service;
    # L=4096, m=64, level-dependent, up/down rate ratio 0.8, jump rates halve per level
    "hessenberg_L4096_m64": dict(kind="banded", L=4096, m=64, p=1, q=4, ratio=0.8, decay=0.5,
                                 seed=5),
    # same recipe at L=32768 (6.4 GB of FP64 blocks): the band waits at the bench's level count
    "hessenberg_L32768_m64": dict(kind="banded", L=32768, m=64, p=1, q=4, ratio=0.8, decay=0.5,
                                  seed=5),
    # jumps +-1, +-2 on L=8192 levels of m=128, paired to 4096 levels of 256
    "penta_L8192_m128": dict(kind="penta", L=8192, m=128, ratio=0.8, scale2=0.3, seed=2),
    # same recipe at L=2048 (1024 paired levels of 256; 1.3 GB per sweep): profiling size
    "penta_L2048_m128": dict(kind="penta", L=2048, m=128, ratio=0.8, scale2=0.3, seed=2),
    # same recipe at L=512 (256 paired levels; L/16): solution parity with the oracle
    "penta_L512_m128": dict(kind="penta", L=512, m=128, ratio=0.8, scale2=0.3, seed=2),
    # same recipe at L=1024 (L/16 of the m=256 chain): solution parity, time to solution
    "qbd_L1024_m256": dict(kind="qbd", L=1024, m=256, ratio=0.9, level_dependent=True, seed=3),
    # L=16384, m=256, level-dependent, ratio 0.9 (FP64 blocks ~25.8 GB)
    "qbd_L16384_m256": dict(kind="qbd", L=16384, m=256, ratio=0.9, level_dependent=True, seed=3),
}


def build(verbose=False):
    """Compile libsynth.so in place (gcc, no FP contraction, OpenMP)."""
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", _SO, _SRC]
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
    u64, i64, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                              ctypes.c_double, ctypes.c_void_p)
    lib.synth_bits.restype = u64
    lib.synth_bits.argtypes = [u64] * 7
    lib.synth_uniform.restype = dbl
    lib.synth_uniform.argtypes = [u64] * 7
    lib.synth_qbd_levels.restype = i32
    lib.synth_qbd_levels.argtypes = [u64, u64, i64, i32, dbl, i32, i64, i64, vp, vp, vp]
    lib.synth_penta_levels.restype = i32
    lib.synth_penta_levels.argtypes = [u64, u64, i64, i32, dbl, dbl, i64, i64, vp, vp, vp]
    lib.synth_qbd_first_irreducible.restype = i32
    lib.synth_banded_levels.restype = i32
    lib.synth_banded_levels.argtypes = [u64, i64, i32, i32, i32, dbl, dbl, i32, i64, i64, vp]
    lib.synth_qbd_first_irreducible.argtypes = [u64, i64, i32, i32, vp, vp, vp]
    _lib = lib
    return lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def uniform(seed, level, kind, i, j, purpose=1, attempt=0):
    """The synthesiser's uniform draw in [0, 1) at one counter coordinate."""
    return _load().synth_uniform(seed, attempt, level, kind, i, j, purpose)


_attempt_cache = {}


def irreducible_attempt(seed, L, m, level_dependent):
    """First redraw index whose QBD generator is irreducible (0 almost always)."""
    key = (seed, L, m, bool(level_dependent))
    if key not in _attempt_cache:
        adj = np.zeros(m * m, np.uint8)
        seen = np.zeros(m, np.uint8)
        stack = np.zeros(m * m + 1, np.int32)
        a = _load().synth_qbd_first_irreducible(seed, L, m, int(level_dependent),
                                                _ptr(adj), _ptr(seen), _ptr(stack))
        if a < 0:
            raise RuntimeError("no irreducible generator within 64 redraws")
        _attempt_cache[key] = a
    return _attempt_cache[key]


def qbd(L, m, ratio, seed, level_dependent=True, l0=0, l1=None, out=None):
    """Generator blocks (dn, loc, up) of levels [l0, l1) of an L-level QBD.

    ``out`` may supply three preallocated C-contiguous float64 arrays of shape
    ``(l1-l0, m, m)`` (e.g. pinned host memory viewed through numpy).
    """
    l1 = L if l1 is None else l1
    n = l1 - l0
    if out is None:
        out = tuple(np.empty((n, m, m), np.float64) for _ in range(3))
    dn, loc, up = out
    att = irreducible_attempt(seed, L, m, level_dependent)
    rc = _load().synth_qbd_levels(seed, att, L, m, float(ratio), int(level_dependent),
                                  l0, l1, _ptr(dn), _ptr(loc), _ptr(up))
    if rc != 0:
        raise ValueError("synth_qbd_levels: bad arguments")
    return dn, loc, up


def penta_paired(L, m, ratio, scale2, seed, J0=0, J1=None, out=None):
    """Block-pentadiagonal generator on L levels of m phases, paired into L/2
    super-levels of 2m phases: returns (dn, loc, up) of super-levels [J0, J1)."""
    J1 = L // 2 if J1 is None else J1
    n, M = J1 - J0, 2 * m
    if out is None:
        out = tuple(np.empty((n, M, M), np.float64) for _ in range(3))
    dn, loc, up = out
    rc = _load().synth_penta_levels(seed, 0, L, m, float(ratio), float(scale2), J0, J1,
                                    _ptr(dn), _ptr(loc), _ptr(up))
    if rc != 0:
        raise ValueError("synth_penta_levels: bad arguments")
    return dn, loc, up


def banded(L, m, p, q, ratio, seed, decay=0.5, level_dependent=True, l0=0, l1=None):
    """Block-banded generator with jumps of -p..q levels (block Hessenberg for
    p == 1 or q == 1): dict {e: (l1-l0, m, m) array of Q[l, l+e]}."""
    l1 = L if l1 is None else l1
    n = l1 - l0
    out = np.empty((p + q + 1, n, m, m), np.float64)
    rc = _load().synth_banded_levels(seed, L, m, p, q, float(ratio), float(decay),
                                     int(level_dependent), l0, l1, _ptr(out))
    if rc != 0:
        raise ValueError("synth_banded_levels: bad arguments")
    return {e: out[e + p] for e in range(-p, q + 1)}


def birth_death(L, lam, mu):
    """m = 1 birth-death generator: up-rate lam, down-rate mu."""
    dn = np.zeros((L, 1, 1))
    up = np.zeros((L, 1, 1))
    loc = np.zeros((L, 1, 1))
    up[:-1] = lam
    dn[1:] = mu
    loc[:, 0, 0] = -(up[:, 0, 0] + dn[:, 0, 0])
    return dn, loc, up


def workload(name, l0=0, l1=None):
    """Blocks of a named workload (levels/super-levels [l0, l1))."""
    w = WORKLOADS[name]
    if w["kind"] == "qbd":
        return qbd(w["L"], w["m"], w["ratio"], w["seed"], w["level_dependent"], l0, l1)
    if w["kind"] == "penta":
        return penta_paired(w["L"], w["m"], w["ratio"], w["scale2"], w["seed"], l0, l1)
    if w["kind"] == "banded":
        return banded(w["L"], w["m"], w["p"], w["q"], w["ratio"], w["seed"], w["decay"], True,
                      l0, l1 if l1 is not None else w["L"])
    if w["kind"] == "birth_death":
        dn, loc, up = birth_death(w["L"], w["lam"], w["mu"])
        l1 = w["L"] if l1 is None else l1
        return dn[l0:l1], loc[l0:l1], up[l0:l1]
    raise KeyError(name)


def workload_shape(name):
    """(levels, block size) of the block-tridiagonal system a workload gives."""
    w = WORKLOADS[name]
    if w["kind"] == "penta":
        return w["L"] // 2, 2 * w["m"]
    return w["L"], w["m"]


REQ_KIND = 7


def request_stream(count=4096, seed=4):
    """Seeded solve requests: L log-uniform in [128, 16384], m uniform over
    {16, 32, 64, 128}, up/down ratio Uniform(0.5, 0.95), level-dependent QBD
    blocks with their own seed.  Arrival gaps are Exp(1) in units of the mean
    inter-arrival time (scale them by the chosen arrival rate)."""
    out = []
    for r in range(count):
        u_l = uniform(seed, r, REQ_KIND, 0, 0)
        u_m = uniform(seed, r, REQ_KIND, 0, 1)
        u_r = uniform(seed, r, REQ_KIND, 0, 2)
        u_a = uniform(seed, r, REQ_KIND, 0, 3)
        L = int(round(128.0 * math.pow(128.0, u_l)))
        L = min(max(L, 128), 16384)
        m = (16, 32, 64, 128)[min(int(u_m * 4), 3)]
        ratio = 0.5 + 0.45 * u_r
        gap = -math.log1p(-u_a)
        out.append(dict(index=r, L=L, m=m, ratio=ratio, seed=1000003 * (seed + 1) + r, gap=gap))
    return out
