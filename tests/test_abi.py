"""The C ABI library loads and exports what include/mc.h declares (CPU only:
only host-side validation paths are called, never GPU work)."""
import ctypes
import os
import subprocess

import pytest

from paper_2302_07551_gb300 import _native as nat
from paper_2302_07551_gb300 import build as pbuild


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(nat.LIB_PATH):
        pbuild.build()
    return nat.load()


def test_every_declared_symbol_is_exported(lib):
    names = nat.declared_functions()
    assert {"mc_create", "mc_factor", "mc_sweep", "mc_solve", "mc_residual", "mc_destroy",
            "mc_workspace_bytes", "mc_status_string"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", nat.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(names) <= exported


def test_workspace_bytes_host_only(lib):
    d = nat.McDesc(64, 8, 1, nat.MC_APPLY_INVERSE, nat.MC_F64)
    n5 = lib.mc_workspace_bytes(ctypes.byref(d))
    d.apply = nat.MC_APPLY_COUPLED
    n7 = lib.mc_workspace_bytes(ctypes.byref(d))
    plane = 64 * 64 * 8      # m*m = 64 is already a multiple of 32 doubles
    assert n7 - n5 == 2 * plane
    assert n5 % 256 == 0
    for bad in [(1, 8, 1, 0, 0), (64, 0, 1, 0, 0), (64, 257, 1, 0, 0), (64, 8, 5, 0, 0),
                (64, 8, 1, 2, 0), (64, 8, 1, 0, 3), (64, 6, 1, 0, 1), (64, 10, 1, 0, 2),
                (64, 8, 3, 0, 1), (64, 32, 1, 0, 0, 1), (64, 64, 4, 0, 0, 1), (64, 64, 1, 0, 0, 2)]:
        assert lib.mc_workspace_bytes(ctypes.byref(nat.McDesc(*bad))) == 0
    # comparison splittings and paired chains
    assert lib.mc_workspace_bytes(ctypes.byref(nat.McDesc(64, 8, 3, 0, 0))) > 0
    assert lib.mc_workspace_bytes(ctypes.byref(nat.McDesc(64, 128, 1, 0, 0, 1))) > 0
    # low-precision storage adds planes and FP32 vectors
    n64 = lib.mc_workspace_bytes(ctypes.byref(nat.McDesc(64, 64, 1, 0, nat.MC_F64)))
    f32 = lib.mc_workspace_bytes(ctypes.byref(nat.McDesc(64, 64, 1, 0, nat.MC_F32)))
    b16 = lib.mc_workspace_bytes(ctypes.byref(nat.McDesc(64, 64, 1, 0, nat.MC_BF16)))
    assert f32 - b16 == 2 * 64 * 64 * 64 * 2      # two planes at 4 vs 2 bytes per entry
    assert b16 > n64
    # padded block stride: m = 5 -> 25 doubles padded to 32
    a = lib.mc_workspace_bytes(ctypes.byref(nat.McDesc(10, 5, 1, 0, 0)))
    b = lib.mc_workspace_bytes(ctypes.byref(nat.McDesc(11, 5, 1, 0, 0)))
    assert b > a


def test_create_rejects_bad_arguments_before_any_gpu_work(lib):
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(1 << 20)
    d = nat.McDesc(64, 8, 1, 0, 0)
    need = lib.mc_workspace_bytes(ctypes.byref(d))
    assert lib.mc_create(ctypes.byref(nat.McDesc(1, 8, 1, 0, 0)), fake, fake, fake, fake, need,
                         None, ctypes.byref(h)) == nat.MC_ERR_ARG
    assert lib.mc_create(ctypes.byref(d), None, fake, fake, fake, need, None,
                         ctypes.byref(h)) == nat.MC_ERR_ARG
    assert lib.mc_create(ctypes.byref(d), ctypes.c_void_p((1 << 20) + 4), fake, fake, fake, need,
                         None, ctypes.byref(h)) == nat.MC_ERR_ARG
    assert lib.mc_create(ctypes.byref(d), fake, fake, fake, fake, need - 8, None,
                         ctypes.byref(h)) == nat.MC_ERR_WORKSPACE
    assert lib.mc_create(ctypes.byref(d), fake, fake, fake, ctypes.c_void_p((1 << 20) + 128),
                         need, None, ctypes.byref(h)) == nat.MC_ERR_WORKSPACE
    assert lib.mc_create(ctypes.byref(d), fake, fake, fake, None, need, None,
                         ctypes.byref(h)) == nat.MC_ERR_WORKSPACE
    assert h.value is None
    for f in ("mc_factor", "mc_sync"):
        assert getattr(lib, f)(None) == nat.MC_ERR_ARG
    assert lib.mc_sweep(None, fake, fake, 1, None) == nat.MC_ERR_ARG
    assert lib.mc_solve(None, None, fake, 1e-12, 0.0, 10, 1, None) == nat.MC_ERR_ARG
    t = nat.McTuning(0, 1)
    assert lib.mc_set_tuning(None, ctypes.byref(t)) == nat.MC_ERR_ARG
    assert lib.mc_get_tuning(None, ctypes.byref(t)) == nat.MC_ERR_ARG
    assert lib.mc_tune(None, fake, 16, ctypes.byref(t), None) == nat.MC_ERR_ARG
    n = ctypes.c_int32()
    assert lib.mc_server_trials(None, None, 0, ctypes.byref(n)) == nat.MC_ERR_ARG
    lib.mc_destroy(None)


def test_status_strings(lib):
    for s in range(0, 9):
        assert lib.mc_status_string(s).decode() not in ("", "unknown status")
    assert lib.mc_status_string(99).decode() == "unknown status"


def test_missing_library_fails_loudly(monkeypatch):
    """Without libmc.so the binding raises: there is no CPU fallback."""
    monkeypatch.setattr(nat, "LIB_PATH", "/nonexistent/libmc.so")
    monkeypatch.setattr(nat, "_lib", None)
    with pytest.raises(ImportError):
        nat.load()
    import paper_2302_07551_gb300 as mc
    with pytest.raises(ImportError):
        mc.Chain.__init__(object.__new__(mc.Chain), *([None] * 3))
