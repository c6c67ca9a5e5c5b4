"""Continuous-batching solve server (mc_server_*): results against the CPU
oracle, bitwise independence of a request from the rest of the batch, the
memory-budget admission, error isolation and autotuning invariance."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

mc = pytest.importorskip("paper_2302_07551_gb300")

MIX = [(40, 16, 0.6), (97, 32, 0.8), (64, 64, 0.7), (33, 128, 0.9), (9, 200, 0.85), (150, 8, 0.5)]


def blocks_for(i, L, m, ratio):
    return synth.qbd(L, m, ratio, seed=500 + i, level_dependent=True)


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_server_results_match_oracle(dtype):
    srv = mc.Server(2 << 30, dtype=dtype, tol=1e-12, check_every=32, autotune=False)
    mix = [x for x in MIX if dtype == "f64" or x[1] % 4 == 0]
    for i, (L, m, ratio) in enumerate(mix):
        assert srv.submit(i, *blocks_for(i, L, m, ratio))
    res = {t: (pi, r, st) for t, pi, r, st in srv.run_until_idle()}
    assert sorted(res) == list(range(len(mix)))
    for i, (L, m, ratio) in enumerate(mix):
        pi, r, st = res[i]
        assert st == 0 and r["converged"] and 0.0 < r["residual"] <= 1e-12
        oc = oracle.Chain(*blocks_for(i, L, m, ratio))
        # the reported residual is the FP64 residual of the returned vector; both
        # sums sit near the rounding floor of Q^T pi (about N u max|Q_ij pi_j|),
        # so they are compared to 1e-14 absolute
        assert abs(r["residual"] - oc.residual(pi)) <= 1e-2 * oc.residual(pi) + 1e-14
        ref = oc.solve(tol=1e-13, maxit=400000, check_every=64)["x"]
        assert rel_l1(pi, ref) <= 1e-10, (i, rel_l1(pi, ref))
    srv.close()


@pytest.mark.parametrize("autotune", [False, True])
@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_server_coupled_stair2_matches_oracle(dtype, autotune):
    """The server in coupled mode with the type-2 stair matrix: each request's
    pi against the oracle's solution (STAIR2 solve of the same chain); tuned,
    the units group levels of the type-2 half-sweeps (the other parity)."""
    srv = mc.Server(2 << 30, dtype=dtype, apply="coupled", stair=2, tol=1e-12, check_every=32,
                    autotune=autotune)
    mix = [(40, 16, 0.6), (64, 64, 0.7), (33, 128, 0.9), (9, 200, 0.85)]
    for i, (L, m, ratio) in enumerate(mix):
        assert srv.submit(i, *blocks_for(i, L, m, ratio))
    res = {t: (pi, r, st) for t, pi, r, st in srv.run_until_idle()}
    for i, (L, m, ratio) in enumerate(mix):
        pi, r, st = res[i]
        assert st == 0 and r["converged"] and r["residual"] <= 1e-12
        oc = oracle.Chain(*blocks_for(i, L, m, ratio))
        ref = oc.solve(tol=1e-13, maxit=400000, check_every=64, method=oracle.STAIR2)["x"]
        assert rel_l1(pi, ref) <= 1e-10, (i, rel_l1(pi, ref))
    srv.close()


@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_same_result_alone_and_in_the_mix(dtype):
    """A request's iterates do not depend on what else is in the batch, when
    the others arrive, or on the launch grid."""
    L, m, ratio = 70, 64, 0.8
    target = blocks_for(99, L, m, ratio)
    alone = mc.Server(1 << 30, dtype=dtype, tol=1e-11, check_every=16, autotune=False)
    alone.submit(7, *target)
    (_, pi_a, r_a, _), = alone.run_until_idle()
    alone.close()
    mix = mc.Server(2 << 30, dtype=dtype, tol=1e-11, check_every=16, autotune=True)
    for i, (Li, mi, ri) in enumerate(MIX[:3]):
        mix.submit(100 + i, *blocks_for(i, Li, mi, ri))
    mix.step()
    mix.submit(7, *target)                     # joins while the others run
    mix.step()
    mix.submit(200, *blocks_for(4, *MIX[4]))   # and more arrive after it
    out = {t: (pi, r) for t, pi, r, st in mix.run_until_idle()}
    pi_m, r_m = out[7]
    assert r_m["sweeps"] == r_a["sweeps"]
    assert np.array_equal(pi_m, pi_a)
    assert r_m["residual"] == r_a["residual"] and 0.0 < r_a["residual"] <= 1e-11
    assert mix.grid()[2] >= 1                  # at least one tuned signature
    mix.close()


def test_admission_by_memory_budget():
    L, m = 64, 64
    probe = mc.Server(64 << 20, tol=1e-10, autotune=False)
    need = probe.request_bytes(L, m)
    probe.close()
    head = 1 << 20                              # request table + outputs
    srv = mc.Server(head + 2 * need + 4096, tol=1e-10, check_every=32, autotune=False)
    b = [blocks_for(i, L, m, 0.7) for i in range(3)]
    assert srv.submit(0, *b[0]) and srv.submit(1, *b[1])
    assert not srv.submit(2, *b[2])             # no room until one retires
    done = []
    while len(done) < 2:
        srv.step()
        while (r := srv.fetch()) is not None:
            done.append(r)
    assert srv.submit(2, *b[2])
    done += srv.run_until_idle()
    assert sorted(t for t, *_ in done) == [0, 1, 2]
    assert all(st == 0 for *_, st in done)
    srv.close()


def test_bad_request_is_isolated():
    srv = mc.Server(1 << 30, tol=1e-12, check_every=32, autotune=False)
    good = blocks_for(1, 50, 16, 0.7)
    dn, loc, up = blocks_for(2, 30, 16, 0.7)
    loc = loc.copy()
    loc[5] = 0.0                                # a level without any rate: zero pivot
    srv.submit(1, *good)
    srv.submit(2, dn, loc, up)
    out = {t: (pi, r, st) for t, pi, r, st in srv.run_until_idle()}
    assert out[2][2] == 4                       # MC_ERR_SINGULAR_BLOCK
    assert out[1][2] == 0 and out[1][1]["converged"]
    ref = oracle.Chain(*good).solve(tol=1e-13, maxit=200000, check_every=32)["x"]
    assert rel_l1(out[1][0], ref) <= 1e-10
    srv.close()


@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_autotuner_search_space_and_invariance(dtype):
    """The autotuner times live chunks over the persistent grid, the levels per
    claimed unit (1, 2, 4 for m > 64; twice that for m <= 64, four times for
    m <= 32), the block-size bucketing and (low precision, small blocks) the
    load depth, keeps one configuration per batch signature, and none of them
    changes a result: every request's pi is bitwise the one of an untuned
    server (whose units already group 2 and 4 levels of the small blocks), and
    matches the oracle."""
    mix = [(300, 16, 0.6), (257, 32, 0.8), (200, 64, 0.7), (120, 128, 0.9), (90, 64, 0.5)]
    out = {}
    for tune in (False, True):
        srv = mc.Server(2 << 30, dtype=dtype, tol=1e-11, check_every=16, autotune=tune)
        for i, (L, m, ratio) in enumerate(mix):
            assert srv.submit(i, *blocks_for(40 + i, L, m, ratio))
        out[tune] = {t: (pi, r, st) for t, pi, r, st in srv.run_until_idle()}
        if tune:
            tr = srv.trials()
            assert {t["levels_per_unit"] for t in tr} >= {1, 2, 4}
            assert {t["split64"] for t in tr} == {0, 1}
            assert {t["blocks_per_sm"] for t in tr} >= {1, 2, 3, 4, 6, 8}
            if dtype != "f64":
                assert {t["deep"] for t in tr} == {0, 1}
            sigs = {t["signature"] for t in tr}
            for sg in sigs:
                assert sum(t["chosen"] for t in tr if t["signature"] == sg) == 1
            assert all(t["sweep_ms"] > 0 and t["sweep_bytes"] > 0 and t["chunk_ms"] >= t["sweep_ms"]
                       for t in tr)
        srv.close()
    for i, (L, m, ratio) in enumerate(mix):
        pi_t, r_t, st_t = out[True][i]
        pi_u, r_u, st_u = out[False][i]
        assert st_t == st_u == 0 and r_t["sweeps"] == r_u["sweeps"]
        assert np.array_equal(pi_t, pi_u), i
        ref = oracle.Chain(*blocks_for(40 + i, L, m, ratio)).solve(
            tol=1e-13, maxit=400000, check_every=64)["x"]
        assert rel_l1(pi_t, ref) <= 1e-10, i
