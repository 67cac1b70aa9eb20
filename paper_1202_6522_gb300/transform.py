"""Torch-tensor front end of libsht: the SHT class and autograd Functions.

PyTorch provides device memory, streams and autograd plumbing only; every step
of every transform runs in libsht's CUDA kernels through the C ABI.

Dtypes select the path: complex128/float64 tensors run the FP64 path,
complex64/float32 tensors the FP32 path.  Spectral tensors are [..., nlm]
complex (packed m-major); grids are [..., nlat, nphi] real, rows north to south.
"""
from __future__ import annotations

import math

import torch

from . import _capi as C


def _next_pow2(v: int) -> int:
    p = 2
    while p < v:
        p *= 2
    return p


class SHT:
    """A Gauss-Legendre spherical harmonic transform plan on one CUDA device."""

    def __init__(self, lmax: int, mmax: int | None = None, nlat: int | None = None,
                 nphi: int | None = None, device=None, fp32_path: str = "f32", fp64_path: str = "f64",
                 mres: int = 1):
        """fp32_path selects how complex64/float32 tensors are transformed:
        "f32" (FP32 recurrence on the CUDA cores), "tc" (tensor cores against
        FP64-built P_n^m panels, split-bf16 products) or "otf" (the same
        contraction with P_n^m generated on the fly, reseeded every 32 degrees
        from FP64 values; scalar transforms, vector ones run "tc").
        fp64_path selects it for complex128/float64 tensors: "f64" (FP64
        recurrence on the CUDA cores) or "tc" (tensor cores on 7-bit digit
        slices of both operands, FP64 accuracy; scalar transforms, lmax <= 1023,
        vector ones run "f64").
        mres > 1 keeps only the orders m = k mres (k <= mmax, mmax mres <= lmax)
        on a grid of one 2 pi / mres sector of longitudes (every path)."""
        self.lmax = int(lmax)
        self.mres = int(mres)
        self.mmax = self.lmax // self.mres if mmax is None else int(mmax)
        self.nlat = self.lmax + 1 if nlat is None else int(nlat)
        self.nphi = max(_next_pow2(2 * self.mmax + 1), 2) if nphi is None else int(nphi)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if fp32_path not in ("f32", "tc", "otf"):
            raise ValueError("fp32_path must be 'f32', 'tc' or 'otf'")
        self.fp32_mode = {"f32": C.SHT_F32, "tc": C.SHT_TC_BF16X3, "otf": C.SHT_TC_OTF}[fp32_path]
        if fp64_path not in ("f64", "tc"):
            raise ValueError("fp64_path must be 'f64' or 'tc'")
        self.fp64_mode = {"f64": C.SHT_F64, "tc": C.SHT_TC_F64}[fp64_path]
        if self.device.type != "cuda":
            raise ValueError("SHT runs on CUDA devices only")
        with torch.cuda.device(self.device):
            self._h = C.sht_create_mres(self.lmax, self.mmax, self.mres, self.nlat, self.nphi)
        self.nlm = C.sht_nlm(self._h)
        x, w = C.sht_gauss(self._h, self.nlat)
        self.x = torch.tensor(x, dtype=torch.float64)
        self.w = torch.tensor(w, dtype=torch.float64)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                torch.cuda.synchronize(self.device)
            except Exception:
                pass
            C.sht_destroy(h)
            self._h = None

    # ------------------------------------------------------------------ helpers
    def lm_index(self, n: int, m: int) -> int:
        return C.sht_lm_index(self._h, n, m)

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def _mode_of(self, t: torch.Tensor) -> int:
        if t.dtype in (torch.complex128, torch.float64):
            return self.fp64_mode
        if t.dtype in (torch.complex64, torch.float32):
            return self.fp32_mode
        raise TypeError(f"unsupported dtype {t.dtype}")

    def _check(self, t: torch.Tensor, kind: str) -> torch.Tensor:
        if t.device != self.device:
            raise ValueError(f"tensor on {t.device}, plan on {self.device}")
        if kind == "spec":
            if not t.is_complex() or t.shape[-1] != self.nlm:
                raise ValueError(f"spectral tensor must be complex [..., {self.nlm}], got {t.dtype} {tuple(t.shape)}")
        else:
            if t.is_complex() or tuple(t.shape[-2:]) != (self.nlat, self.nphi):
                raise ValueError(f"grid tensor must be real [..., {self.nlat}, {self.nphi}], got {tuple(t.shape)}")
        return t.contiguous()

    def _grid_like(self, spec: torch.Tensor) -> torch.Tensor:
        dt = torch.float64 if spec.dtype == torch.complex128 else torch.float32
        return torch.empty(spec.shape[:-1] + (self.nlat, self.nphi), dtype=dt, device=self.device)

    def _spec_like(self, grid: torch.Tensor) -> torch.Tensor:
        dt = torch.complex128 if grid.dtype == torch.float64 else torch.complex64
        return torch.empty(grid.shape[:-2] + (self.nlm,), dtype=dt, device=self.device)

    # ------------------------------------------------------- raw (no autograd)
    def synth_(self, spec):
        spec = self._check(spec, "spec")
        out = self._grid_like(spec)
        b = max(1, math.prod(spec.shape[:-1]))
        C.sht_synth(self._h, spec.data_ptr(), out.data_ptr(), b, self._mode_of(spec), self._stream())
        return out

    def analys_(self, grid):
        grid = self._check(grid, "grid")
        out = self._spec_like(grid)
        b = max(1, math.prod(grid.shape[:-2]))
        C.sht_analys(self._h, grid.data_ptr(), out.data_ptr(), b, self._mode_of(grid), self._stream())
        return out

    def synth_adj_(self, grid):
        grid = self._check(grid, "grid")
        out = self._spec_like(grid)
        b = max(1, math.prod(grid.shape[:-2]))
        C.sht_synth_adj(self._h, grid.data_ptr(), out.data_ptr(), b, self._mode_of(grid), self._stream())
        return out

    def analys_adj_(self, spec):
        spec = self._check(spec, "spec")
        out = self._grid_like(spec)
        b = max(1, math.prod(spec.shape[:-1]))
        C.sht_analys_adj(self._h, spec.data_ptr(), out.data_ptr(), b, self._mode_of(spec), self._stream())
        return out

    def synth_vec_(self, S, T):
        S = self._check(S, "spec")
        T = self._check(T, "spec")
        if S.shape != T.shape or S.dtype != T.dtype:
            raise ValueError("S and T must have the same shape and dtype")
        vt, vp = self._grid_like(S), self._grid_like(S)
        b = max(1, math.prod(S.shape[:-1]))
        C.sht_synth_vec(self._h, S.data_ptr(), T.data_ptr(), vt.data_ptr(), vp.data_ptr(), b,
                        self._mode_of(S), self._stream())
        return vt, vp

    def analys_vec_(self, vt, vp):
        vt = self._check(vt, "grid")
        vp = self._check(vp, "grid")
        if vt.shape != vp.shape or vt.dtype != vp.dtype:
            raise ValueError("v_theta and v_phi must have the same shape and dtype")
        S, T = self._spec_like(vt), self._spec_like(vt)
        b = max(1, math.prod(vt.shape[:-2]))
        C.sht_analys_vec(self._h, vt.data_ptr(), vp.data_ptr(), S.data_ptr(), T.data_ptr(), b,
                         self._mode_of(vt), self._stream())
        return S, T

    def synth_vec_adj_(self, gt, gp):
        gt = self._check(gt, "grid")
        gp = self._check(gp, "grid")
        S, T = self._spec_like(gt), self._spec_like(gt)
        b = max(1, math.prod(gt.shape[:-2]))
        C.sht_synth_vec_adj(self._h, gt.data_ptr(), gp.data_ptr(), S.data_ptr(), T.data_ptr(), b,
                            self._mode_of(gt), self._stream())
        return S, T

    def analys_vec_adj_(self, S, T):
        S = self._check(S, "spec")
        T = self._check(T, "spec")
        gt, gp = self._grid_like(S), self._grid_like(S)
        b = max(1, math.prod(S.shape[:-1]))
        C.sht_analys_vec_adj(self._h, S.data_ptr(), T.data_ptr(), gt.data_ptr(), gp.data_ptr(), b,
                             self._mode_of(S), self._stream())
        return gt, gp

    # ---------------------------------------------------- differentiable API
    def synth(self, spec):
        """Scalar synthesis (Sec. 2.2); differentiable (backward = sht_synth_adj)."""
        return _Synth.apply(self, spec)

    def analys(self, grid):
        """Scalar analysis (Sec. 2.3); differentiable (backward = sht_analys_adj)."""
        return _Analys.apply(self, grid)

    def synth_vec(self, S, T):
        """Spheroidal/toroidal synthesis; differentiable."""
        return _SynthVec.apply(self, S, T)

    def analys_vec(self, vt, vp):
        """Spheroidal/toroidal analysis; differentiable."""
        return _AnalysVec.apply(self, vt, vp)

    def sync_status(self):
        return C.sht_sync_status(self._h, self._stream())


class _Synth(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sht, spec):
        ctx.sht = sht
        return sht.synth_(spec)

    @staticmethod
    def backward(ctx, g):
        return None, ctx.sht.synth_adj_(g)


class _Analys(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sht, grid):
        ctx.sht = sht
        return sht.analys_(grid)

    @staticmethod
    def backward(ctx, g):
        return None, ctx.sht.analys_adj_(g)


class _SynthVec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sht, S, T):
        ctx.sht = sht
        return sht.synth_vec_(S, T)

    @staticmethod
    def backward(ctx, gt, gp):
        sht = ctx.sht
        if gt is None:
            gt = torch.zeros_like(gp)
        if gp is None:
            gp = torch.zeros_like(gt)
        S, T = sht.synth_vec_adj_(gt, gp)
        return None, S, T


class _AnalysVec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sht, vt, vp):
        ctx.sht = sht
        return sht.analys_vec_(vt, vp)

    @staticmethod
    def backward(ctx, gS, gT):
        sht = ctx.sht
        if gS is None:
            gS = torch.zeros_like(gT)
        if gT is None:
            gT = torch.zeros_like(gS)
        gt, gp = sht.analys_vec_adj_(gS, gT)
        return None, gt, gp


class UnevenBatch:
    """Many FP32 scalar fields of different truncations transformed by one
    graph launch.  path="f32": persistent CUDA-core kernels over a
    longest-first tile list; "tc": one batched tensor-core contraction per
    group of equal shape; "auto": both timed at construction, the faster kept
    (``self.path`` tells which, ``self.tuned_ms`` the two times)."""

    _PATHS = {"f32": C.SHT_F32, "tc": C.SHT_TC_BF16X3, "auto": C.SHT_F32_AUTO}

    def __init__(self, lmax, nlat=None, nphi=None, device=None, use_graph=True, path="f32"):
        self.lmax = [int(v) for v in lmax]
        self.nlat = [l + 1 for l in self.lmax] if nlat is None else [int(v) for v in nlat]
        self.nphi = ([max(_next_pow2(2 * l + 1), 2) for l in self.lmax] if nphi is None
                     else [int(v) for v in nphi])
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.use_graph = use_graph
        if path not in self._PATHS:
            raise ValueError("path must be 'f32', 'tc' or 'auto'")
        with torch.cuda.device(self.device):
            self._h = C.sht_batch_create_mode(self.lmax, self.nlat, self.nphi, self._PATHS[path])
        mode, ms_f32, ms_tc = C.sht_batch_mode(self._h)
        self.path = "tc" if mode == C.SHT_TC_BF16X3 else "f32"
        self.tuned_ms = {"f32": ms_f32, "tc": ms_tc} if path == "auto" else None
        self.nlm = [(l + 1) * (l + 2) // 2 for l in self.lmax]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            C.sht_batch_destroy(h)
            self._h = None

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def synth_(self, specs, out=None):
        """specs: list of complex64 [nlm_f] tensors -> list of float32 [nlat_f, nphi_f]."""
        specs = [s.contiguous() for s in specs]
        for s, n in zip(specs, self.nlm):
            if s.dtype != torch.complex64 or s.numel() != n or s.device != self.device:
                raise ValueError("each spectrum must be complex64 [nlm_f] on the batch's device")
        if out is None:
            out = [torch.empty(la, ph, dtype=torch.float32, device=self.device) for la, ph in zip(self.nlat, self.nphi)]
        C.sht_batch_synth(self._h, [s.data_ptr() for s in specs], [g.data_ptr() for g in out],
                          self.use_graph, self._stream())
        return out

    def analys_(self, grids, out=None):
        grids = [g.contiguous() for g in grids]
        for g, la, ph in zip(grids, self.nlat, self.nphi):
            if g.dtype != torch.float32 or tuple(g.shape) != (la, ph) or g.device != self.device:
                raise ValueError("each grid must be float32 [nlat_f, nphi_f] on the batch's device")
        if out is None:
            out = [torch.empty(n, dtype=torch.complex64, device=self.device) for n in self.nlm]
        C.sht_batch_analys(self._h, [g.data_ptr() for g in grids], [s.data_ptr() for s in out],
                           self.use_graph, self._stream())
        return out
