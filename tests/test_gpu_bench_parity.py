"""GPU path vs the CPU oracle at the benchmark's sizes and launch configuration.

* Iterates: K = 50 sweeps from the uniform vector on the full 32768-level,
  m = 64 chain (one fused launch, the benchmark's grid), compared with the
  oracle over the whole vector: relative L1 <= 1e-12, and e^T z / step error
  of the last sweep.
* Solutions: each side runs to its own residual ||Q^T pi||_1 <= 1e-12 with the
  same check interval; the two stationary vectors agree to relative L1
  <= 1e-10.  Chains: the same recipes as the three FP64 bench chains at L/16
  (2048 levels of 64; 1024 levels of 256; the pentadiagonal chain on 512
  levels of 128 paired into 256 levels of 256), and the m = 256 chain in FP32
  and BF16 mixed-precision refinement, whose error against the FP64 oracle is
  printed (pytest -s) beside the assertion.

The oracle solutions take tens of seconds to minutes of host time each, so
they are computed once per module.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

mc = pytest.importorskip("paper_2302_07551_gb300")

TOL = 1e-12
CHECK = 64


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l1(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_full_size_50_sweeps_from_uniform_qbd_L32768_m64():
    name = "qbd_L32768_m64"
    L, m = synth.workload_shape(name)
    N = L * m
    K = 50
    blocks = synth.workload(name)
    ch = mc.Chain(*(dev(b) for b in blocks))
    oc = oracle.Chain(*blocks)
    del blocks
    x0 = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    stats = torch.zeros(3, dtype=torch.float64, device="cuda")
    x = ch.sweep(x0, nsweeps=K, stats=stats).cpu().numpy()
    ch.close()
    u = np.full(N, 1.0 / N)
    prev = oc.sweeps(u, K - 1)
    ref, s, d = oc.normalised_sweep(prev)
    err = rel_l1(x, ref)
    print(f"\n{name}: {K} sweeps from uniform, GPU vs oracle relative L1 {err:.3e}")
    assert err <= 1e-12
    st = stats.cpu().numpy()
    assert abs(st[0] - s) <= 1e-12 * abs(s)
    assert abs(st[1] - d) <= 1e-12
    assert (x >= 0).all() and abs(x.sum() - 1.0) <= 1e-12


_ORACLE = {}


def oracle_solution(name):
    """The oracle's stationary vector of a workload (residual <= TOL)."""
    if name not in _ORACLE:
        oc = oracle.Chain(*synth.workload(name))
        r = oc.solve(tol=TOL, maxit=5_000_000, check_every=CHECK, history=False)
        assert r["resid"] <= TOL
        _ORACLE[name] = r
    return _ORACLE[name]


@pytest.mark.parametrize("name,dtype,apply", [
    ("qbd_L2048_m64", "f64", "inverse"),
    ("penta_L512_m128", "f64", "inverse"),
    ("qbd_L1024_m256", "f64", "inverse"),
    ("qbd_L1024_m256", "f64", "coupled"),
    ("qbd_L1024_m256", "f32", "inverse"),
    ("qbd_L1024_m256", "bf16", "coupled"),
])
def test_solution_parity_reduced_bench_chains(name, dtype, apply):
    ref = oracle_solution(name)
    paired = synth.WORKLOADS[name]["kind"] == "penta" and dtype == "f64" and apply == "inverse"
    ch = mc.Chain(*(dev(b) for b in synth.workload(name)), dtype=dtype, apply=apply,
                  paired=paired)
    pi, res = ch.solve(tol=TOL, maxit=5_000_000, check_every=CHECK)
    ch.close()
    pi = pi.cpu().numpy()
    err = rel_l1(pi, ref["x"])
    print(f"\n{name} {dtype} {apply}: GPU {res['sweeps']} sweeps, residual {res['residual']:.3e}; "
          f"oracle {ref['sweeps']} sweeps, residual {ref['resid']:.3e}; relative L1 {err:.3e}")
    assert res["converged"] and res["residual"] <= TOL
    assert err <= 1e-10
    assert (pi >= 0).all() and abs(pi.sum() - 1.0) <= 1e-12
    if dtype == "f64":
        # same iteration, same check interval: the same stopping check
        assert res["sweeps"] == ref["sweeps"]
