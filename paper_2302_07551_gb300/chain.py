"""Torch-facing wrapper of one libmc chain handle (argument marshalling only)."""
import ctypes

import torch

from . import _native as nat


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _need(t, shape=None, name="tensor"):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


class Chain:
    """A block-tridiagonal chain resident on the GPU.

    dn, loc, up: float64 CUDA tensors (L, m, m), generator blocks of Q
    (row-major): dn[l] = Q[l, l-1], loc[l] = Q[l, l], up[l] = Q[l, l+1].
    stair: 1 or 2 (stair matrix type).  apply: "inverse" or "coupled".
    dtype: "f64" (plain FP64 iteration) or "f32" / "bf16" (mixed-precision
    refinement in solve(); check_every = correction sweeps per outer step).
    The library copies the blocks into its workspace (a torch uint8 tensor
    owned by this object); the inputs may be freed after construction.
    """

    def __init__(self, dn, loc, up, stair=1, apply="inverse", stream=None, factor=True,
                 dtype="f64", paired=False, diags=None):
        lib = nat.load()
        if diags is not None:
            # block-banded: diags = {e: (L, m, m) tensor of Q[l, l+e]}
            lower, upper = -min(diags), max(diags)
            loc = diags[0]
            for e, t in diags.items():
                _need(t, loc.shape, f"diags[{e}]")
        else:
            lower = upper = 1
            for t, n in ((dn, "dn"), (loc, "loc"), (up, "up")):
                _need(t, loc.shape, n)
        L, m, _ = loc.shape
        self.L, self.m, self.N = int(L), int(m), int(L) * int(m)
        self.device = loc.device
        self.desc = nat.McDesc(self.L, self.m, int(stair),
                               nat.MC_APPLY_COUPLED if apply == "coupled" else nat.MC_APPLY_INVERSE,
                               nat.DTYPES[dtype], 1 if paired else 0, lower, upper)
        self.dtype = dtype
        self.apply = apply
        nbytes = lib.mc_workspace_bytes(ctypes.byref(self.desc))
        if nbytes == 0:
            raise ValueError("invalid chain description")
        self.ws_bytes = nbytes
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        if diags is not None:
            arr = (ctypes.c_void_p * (lower + upper + 1))(
                *[diags[e].data_ptr() for e in range(-lower, upper + 1)])
            nat.check(lib.mc_create_banded(ctypes.byref(self.desc), arr,
                                           ctypes.c_void_p(self._ws_ptr), nbytes,
                                           ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.byref(h)), "mc_create_banded")
        else:
            nat.check(lib.mc_create(ctypes.byref(self.desc), _ptr(dn), _ptr(loc), _ptr(up),
                                    ctypes.c_void_p(self._ws_ptr), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                      "mc_create")
        self._h = h
        self._lib = lib
        if factor:
            self.factor()

    # --- entry points -------------------------------------------------------
    def factor(self):
        nat.check(self._lib.mc_factor(self._h), "mc_factor")

    def sweep(self, x_in, x_out=None, nsweeps=1, stats=None):
        """nsweeps normalised staircase sweeps (async on the chain's stream)."""
        _need(x_in, (self.N,), "x_in")
        if x_out is None:
            x_out = torch.empty_like(x_in)
        _need(x_out, (self.N,), "x_out")
        sp = None
        if stats is not None:
            _need(stats, (3,), "stats")
            sp = _ptr(stats)
        nat.check(self._lib.mc_sweep(self._h, _ptr(x_in), _ptr(x_out), int(nsweeps), sp), "mc_sweep")
        return x_out

    def profile(self, x_in, x_out=None, nsweeps=1):
        """mc_profile: sweeps with per-kernel CUDA events; returns (x_out,
        dict of summed milliseconds per kernel kind and launch count)."""
        _need(x_in, (self.N,), "x_in")
        if x_out is None:
            x_out = torch.empty_like(x_in)
        ms = (ctypes.c_double * 5)()
        nat.check(self._lib.mc_profile(self._h, _ptr(x_in), _ptr(x_out), int(nsweeps), ms),
                  "mc_profile")
        return x_out, dict(fused=ms[4] == 1.0, sweeps_ms=ms[0], scale_ms=ms[1], norm_ms=ms[2],
                           launches=int(ms[3]))

    def sweep_host(self, x_in, x_out, nsweeps=1, stats=True):
        """Host-buffer variant (x_in, x_out: CPU float64, ideally pinned).
        Returns [e^T z, step, residual] (stats=True) or None (stats=False:
        no residual is formed)."""
        for t in (x_in, x_out):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != self.N:
                raise ValueError("host vectors must be contiguous float64 CPU tensors of length N")
        st = (ctypes.c_double * 3)() if stats else None
        nat.check(self._lib.mc_sweep_host(self._h, _ptr(x_in), _ptr(x_out), int(nsweeps), st),
                  "mc_sweep_host")
        return list(st) if stats else None

    def solve(self, x0=None, tol=1e-12, eps=0.0, maxit=1_000_000, check_every=32, pi=None,
              raise_on_maxit=True):
        """Iterate to ||Q^T pi||_1 <= tol (or step <= eps); returns (pi, result dict)."""
        if pi is None:
            pi = torch.empty(self.N, dtype=torch.float64, device=self.device)
        _need(pi, (self.N,), "pi")
        x0p = None
        if x0 is not None:
            _need(x0, (self.N,), "x0")
            x0p = _ptr(x0)
        res = nat.McResult()
        rc = self._lib.mc_solve(self._h, x0p, _ptr(pi), float(tol), float(eps), int(maxit),
                                int(check_every), ctypes.byref(res))
        out = dict(sweeps=res.sweeps, residual=res.residual_l1, step=res.step_l1,
                   contraction=res.contraction, converged=bool(res.converged), status=rc)
        if rc != nat.MC_OK and not (rc == nat.MC_ERR_NO_CONVERGENCE and not raise_on_maxit):
            raise nat.McError(rc, "mc_solve")
        return pi, out

    def residual(self, pi):
        _need(pi, (self.N,), "pi")
        r = ctypes.c_double()
        nat.check(self._lib.mc_residual(self._h, _ptr(pi), ctypes.byref(r)), "mc_residual")
        return r.value

    def export(self, plane, level0=0, count=None):
        """Stored blocks as a (count, m, m) tensor; block[j, i] is entry (i, j)
        of the Q^T block (column-major storage, see include/mc.h)."""
        count = self.L - level0 if count is None else count
        out = torch.empty((count, self.m, self.m), dtype=torch.float64, device=self.device)
        nat.check(self._lib.mc_export(self._h, nat.PLANES[plane], int(level0), int(count),
                                      _ptr(out)), "mc_export")
        return out

    def tune(self, x, nsweeps=64):
        """mc_tune: time the fused launch configurations on nsweeps sweeps
        from x (a CUDA float64 vector, only read) and keep the fastest;
        returns (blocks_per_sm, levels_per_unit, milliseconds)."""
        _need(x, (self.N,), "x")
        t = nat.McTuning()
        ms = ctypes.c_double()
        nat.check(self._lib.mc_tune(self._h, _ptr(x), int(nsweeps), ctypes.byref(t),
                                    ctypes.byref(ms)), "mc_tune")
        return t.blocks_per_sm, t.levels_per_unit, ms.value

    def set_tuning(self, blocks_per_sm=0, levels_per_unit=1):
        nat.check(self._lib.mc_set_tuning(self._h, ctypes.byref(
            nat.McTuning(int(blocks_per_sm), int(levels_per_unit)))), "mc_set_tuning")

    def tuning(self):
        t = nat.McTuning()
        nat.check(self._lib.mc_get_tuning(self._h, ctypes.byref(t)), "mc_get_tuning")
        return t.blocks_per_sm, t.levels_per_unit

    def sync(self):
        nat.check(self._lib.mc_sync(self._h), "mc_sync")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @classmethod
    def banded(cls, diags, **kw):
        """Block-banded chain from {e: (L, m, m) float64 CUDA tensor of Q[l, l+e]}."""
        return cls(None, None, None, diags=diags, **kw)


def solve(dn, loc, up, tol=1e-12, **kw):
    """One-shot: build, factor and solve; returns (pi, result)."""
    stair = kw.pop("stair", 1)
    apply = kw.pop("apply", "inverse")
    ch = Chain(dn, loc, up, stair=stair, apply=apply)
    try:
        return ch.solve(tol=tol, **kw)
    finally:
        ch.close()
