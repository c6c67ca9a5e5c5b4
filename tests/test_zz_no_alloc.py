"""mc_residual_noalloc: the direct residual for callers that cannot allocate
device memory (inside a graph capture, under another allocator's budget, or
holding only borrowed device pointers).  It must agree with mc_residual, the
workspace-based entry point, and with the CPU oracle's direct residual, on two
calls in a row (the second call reuses the library's static scratch left
behind by the first), for every register-tile width of the kernel (m = 1 to
256) and at the scratch capacity L = 65536."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,m", [(300, 1), (300, 33), (300, 40), (120, 100), (64, 256),
                                 (65536, 8)])
def test_noalloc_residual_matches_workspace_residual_twice(L, m):
    torch = pytest.importorskip("torch")
    import paper_2302_07551_gb300 as mc
    from paper_2302_07551_gb300 import _native as nat

    lib = nat.load()
    host = synth.qbd(L, m, 0.85, seed=12 + m)
    blocks = [torch.from_numpy(b).cuda() for b in host]
    oc = oracle.Chain(*host)
    ch = mc.Chain(*blocks)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(3 + m)
    for call in range(2):
        x = rng.random(L * m) * (call + 1)
        pi = torch.from_numpy(x).cuda()
        ref = ch.residual(pi)
        want = oc.residual(x)
        torch.cuda.synchronize()
        rc = lib.mc_residual_noalloc(*(ctypes.c_void_p(b.data_ptr()) for b in blocks), L, m,
                                     ctypes.c_void_p(pi.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), None)
        assert rc == nat.MC_OK
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)
        assert abs(got - want) <= 1e-12 * want, (call, got, want)
    # sizes beyond the scratch capacity are refused before any GPU work
    fake = ctypes.c_void_p(1 << 20)
    assert lib.mc_residual_noalloc(fake, fake, fake, (1 << 16) + 1, 8, fake, fake,
                                   None) == nat.MC_ERR_ARG
    assert lib.mc_residual_noalloc(fake, fake, fake, 1, 8, fake, fake, None) == nat.MC_ERR_ARG
    assert lib.mc_residual_noalloc(fake, fake, fake, 8, 257, fake, fake, None) == nat.MC_ERR_ARG
    ch.close()
