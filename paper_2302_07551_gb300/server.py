"""Torch-facing wrapper of the continuous-batching solve server (mc_server_*).

Argument marshalling only: admission, batching, sweeps, convergence checks and
retirement all happen in libmc.  The arena is one torch uint8 CUDA tensor
owned by this object (the library itself never allocates device memory).
"""
import ctypes

import numpy as np
import torch

from . import _native as nat


class Server:
    def __init__(self, arena_bytes, dtype="f64", apply="inverse", stair=1, check_every=32,
                 tol=1e-10, maxit=10_000_000, max_active=256, autotune=True, stream=None,
                 device="cuda"):
        self._lib = nat.load()
        self.device = torch.device(device)
        self._arena = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device=self.device)
        ptr = (self._arena.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.desc = nat.McServerDesc(nat.DTYPES[dtype],
                                     nat.MC_APPLY_COUPLED if apply == "coupled" else nat.MC_APPLY_INVERSE,
                                     int(stair), int(check_every), float(tol), int(maxit),
                                     int(max_active), 1 if autotune else 0)
        h = ctypes.c_void_p()
        torch.cuda.synchronize(self.device)
        nat.check(self._lib.mc_server_create(ctypes.byref(self.desc), ctypes.c_void_p(ptr),
                                             int(arena_bytes),
                                             ctypes.c_void_p(self.stream.cuda_stream),
                                             ctypes.byref(h)), "mc_server_create")
        self._h = h
        self._keep = {}

    def request_bytes(self, L, m):
        return self._lib.mc_server_request_bytes(self._h, int(L), int(m))

    def submit(self, tag, dn, loc, up):
        """Admit a request (host float64 arrays (L, m, m)); False if no room now."""
        L, m, _ = loc.shape
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (dn, loc, up)]
        rc = self._lib.mc_server_submit(self._h, int(tag), int(L), int(m),
                                        *(ctypes.c_void_p(a.ctypes.data) for a in arrs))
        if rc == nat.MC_ERR_WORKSPACE:
            return False
        nat.check(rc, "mc_server_submit")
        self._keep[int(tag)] = int(L) * int(m)
        return True

    def step(self):
        na, nd = ctypes.c_int32(), ctypes.c_int32()
        nat.check(self._lib.mc_server_step(self._h, ctypes.byref(na), ctypes.byref(nd)),
                  "mc_server_step")
        return na.value, nd.value

    def fetch(self):
        """Oldest finished request as (tag, pi, result dict, status), or None."""
        if not self._keep:
            return None
        cap = max(self._keep.values())
        pi = np.full(cap, np.nan)      # stays NaN if the result could not be copied out
        tag = ctypes.c_int64()
        res = nat.McResult()
        st = ctypes.c_int32()
        rc = self._lib.mc_server_fetch(self._h, ctypes.byref(tag), ctypes.c_void_p(pi.ctypes.data),
                                       cap, ctypes.byref(res), ctypes.byref(st))
        if rc == nat.MC_ERR_ARG:
            return None
        nat.check(rc, "mc_server_fetch")
        n = self._keep.pop(tag.value)
        return tag.value, pi[:n].copy(), dict(sweeps=res.sweeps, residual=res.residual_l1,
                                              step=res.step_l1, contraction=res.contraction,
                                              converged=bool(res.converged)), st.value

    def grid(self):
        b, t, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        nat.check(self._lib.mc_server_grid(self._h, ctypes.byref(b), ctypes.byref(t),
                                           ctypes.byref(n)), "mc_server_grid")
        return b.value, t.value, n.value

    def trials(self):
        """The autotuner's timed chunks: one dict per candidate configuration
        (signature, blocks per SM, levels per unit, bucketing, load depth,
        whether it was kept, chunk and sweep-launch milliseconds, algorithmic
        bytes of the sweep launches)."""
        n = ctypes.c_int32()
        nat.check(self._lib.mc_server_trials(self._h, None, 0, ctypes.byref(n)),
                  "mc_server_trials")
        arr = (nat.McServerTuning * max(n.value, 1))()
        nat.check(self._lib.mc_server_trials(self._h, arr, n.value, ctypes.byref(n)),
                  "mc_server_trials")
        return [dict(signature=t.signature, blocks_per_sm=t.blocks_per_sm,
                     levels_per_unit=t.levels_per_unit, split64=t.split64, deep=t.deep,
                     chosen=bool(t.chosen), chunk_ms=t.chunk_ms, sweep_ms=t.sweep_ms,
                     sweep_bytes=t.sweep_bytes) for t in arr[:n.value]]

    def run_until_idle(self):
        """Step until no request is active; returns all finished results."""
        out = []
        while True:
            na, _ = self.step()
            while True:
                r = self.fetch()
                if r is None:
                    break
                out.append(r)
            if na == 0:
                return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
