"""PyTorch-facing wrappers of the C ABI (device memory and streams only).

``Advect`` owns one library context for a grid shape and element type and
calls it on torch tensors (CUDA, contiguous, layout ``(nx, ny, nz)``) on the
current torch stream.  ``AdvectFn`` is the ``torch.autograd.Function`` whose
backward is the library's gather-form adjoint.  No arithmetic of the method
happens here.
"""
from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable

from . import _abi

_DTYPES = {"f64": (_abi.ADVECT_F64, torch.float64), "f32": (_abi.ADVECT_F32, torch.float32),
           "f16s": (_abi.ADVECT_F16S, torch.float16), "f64ff": (_abi.ADVECT_F64_FF, torch.float64)}


def coefficients_from_grid(grid):
    """Library coefficient setup from an object with nz, dx, dy, z, zn, rho, rhon."""
    return _abi.advect_coeffs_from_grid(grid.nz, grid.dx, grid.dy, grid.z, grid.zn, grid.rho,
                                        grid.rhon)


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Advect:
    """A library context for one (nx, ny, nz) grid and element type."""

    def __init__(self, nx, ny, nz, coeffs, dtype="f64", f64_levels=None):
        if dtype not in _DTYPES:
            raise ValueError(f"dtype must be one of {sorted(_DTYPES)}")
        self.shape = (int(nx), int(ny), int(nz))
        self.dtype_name = dtype
        self.code, self.torch_dtype = _DTYPES[dtype]
        self.coeffs = coeffs
        self.handle = _abi.advect_create(nx, ny, nz, coeffs, self.code)
        if f64_levels is not None:
            _abi.advect_set_f64_levels(self.handle, f64_levels)

    # -- helpers --------------------------------------------------------
    def _check(self, *ts):
        for t in ts:
            if not isinstance(t, torch.Tensor):
                raise TypeError("expected torch tensors")
            if tuple(t.shape) != self.shape or t.dtype != self.torch_dtype:
                raise ValueError(f"expected shape {self.shape} and dtype {self.torch_dtype}, got "
                                 f"{tuple(t.shape)} {t.dtype}")
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("tensors must be contiguous CUDA tensors")

    def empty(self):
        return torch.empty(self.shape, dtype=self.torch_dtype, device="cuda")

    def kernel_name(self, adjoint=False):
        return _abi.advect_kernel_name(self.handle, adjoint)

    def autotune(self, enable=True):
        _abi.advect_autotune(self.handle, enable)

    def tuned_config(self, adjoint=False):
        return _abi.advect_tuned_config(self.handle, adjoint)

    def output_scales(self, in_scales):
        return _abi.advect_f16s_output_scales(self.handle, in_scales)

    # -- calls ----------------------------------------------------------
    def forward(self, u, v, w, out=None, scales=None):
        self._check(u, v, w)
        su, sv, sw = out if out is not None else (self.empty(), self.empty(), self.empty())
        self._check(su, sv, sw)
        _abi.advect_forward(self.handle, u.data_ptr(), v.data_ptr(), w.data_ptr(), su.data_ptr(),
                            sv.data_ptr(), sw.data_ptr(), scales, _stream())
        return su, sv, sw

    def integrate(self, u, v, w, dt, base=None, out=None, scales=None):
        """(base + dt * su, base + dt * sv, base + dt * sw) in one kernel; base
        defaults to (u, v, w).  out may be base itself (in-place step)."""
        self._check(u, v, w)
        if base is not None:
            self._check(*base)
        uo, vo, wo = out if out is not None else (self.empty(), self.empty(), self.empty())
        self._check(uo, vo, wo)
        bp = [b.data_ptr() for b in base] if base is not None else [None] * 3
        _abi.advect_forward_integrate(self.handle, u.data_ptr(), v.data_ptr(), w.data_ptr(), *bp, dt,
                                      uo.data_ptr(), vo.data_ptr(), wo.data_ptr(), scales, _stream())
        return uo, vo, wo

    def adjoint(self, u, v, w, dsu, dsv, dsw, out=None):
        self._check(u, v, w, dsu, dsv, dsw)
        du, dv, dw = out if out is not None else (self.empty(), self.empty(), self.empty())
        self._check(du, dv, dw)
        _abi.advect_adjoint(self.handle, u.data_ptr(), v.data_ptr(), w.data_ptr(), dsu.data_ptr(),
                            dsv.data_ptr(), dsw.data_ptr(), du.data_ptr(), dv.data_ptr(),
                            dw.data_ptr(), _stream())
        return du, dv, dw

    def forward_host(self, u, v, w, out, scales=None):
        """Host buffers (CPU tensors, pinned for full copy speed) in and out."""
        ts = [u, v, w, *out]
        for t in ts:
            if t.is_cuda or not t.is_contiguous() or tuple(t.shape) != self.shape \
                    or t.dtype != self.torch_dtype:
                raise ValueError("forward_host takes contiguous CPU tensors of the context's shape/dtype")
        _abi.advect_forward_host(self.handle, *(t.data_ptr() for t in ts), scales)
        return out

    def sync(self):
        _abi.advect_sync(self.handle, _stream())

    def close(self):
        if self.handle:
            _abi.advect_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AdvectFn(torch.autograd.Function):
    """(u, v, w) -> (su, sv, sw) with the library's adjoint as backward."""

    @staticmethod
    def forward(ctx, u, v, w, op: Advect):
        u, v, w = u.contiguous(), v.contiguous(), w.contiguous()
        su, sv, sw = op.forward(u, v, w)
        ctx.save_for_backward(u, v, w)
        ctx.op = op
        return su, sv, sw

    @staticmethod
    @once_differentiable
    def backward(ctx, dsu, dsv, dsw):
        u, v, w = ctx.saved_tensors
        op = ctx.op
        z = None
        grads = []
        for g in (dsu, dsv, dsw):
            if g is None:
                z = z if z is not None else torch.zeros_like(u)
                g = z
            grads.append(g.contiguous())
        du, dv, dw = op.adjoint(u, v, w, *grads)
        return du, dv, dw, None


def advect(u, v, w, op: Advect):
    """Differentiable PW advection: returns (su, sv, sw)."""
    return AdvectFn.apply(u, v, w, op)


class AdvectEnsemble:
    """Several grids of uneven shape, run in one persistent launch."""

    def __init__(self, shapes, coeffs_list, dtype="f32"):
        if dtype not in ("f64", "f32"):
            raise ValueError("ensembles support f64 and f32")
        self.shapes = [tuple(int(x) for x in s) for s in shapes]
        self.code, self.torch_dtype = _DTYPES[dtype]
        self.handle = _abi.advect_ensemble_create(self.shapes, coeffs_list, self.code)

    def _ptrs(self, ts):
        if len(ts) != len(self.shapes):
            raise ValueError("one tensor per member expected")
        for t, s in zip(ts, self.shapes):
            if tuple(t.shape) != s or t.dtype != self.torch_dtype or not t.is_cuda or not t.is_contiguous():
                raise ValueError("member tensors must be contiguous CUDA tensors of the member's shape")
        return [t.data_ptr() for t in ts]

    def empty(self):
        return [torch.empty(s, dtype=self.torch_dtype, device="cuda") for s in self.shapes]

    def forward(self, u, v, w, out=None):
        su, sv, sw = out if out is not None else (self.empty(), self.empty(), self.empty())
        _abi.advect_ensemble_forward(self.handle, *(self._ptrs(x) for x in (u, v, w, su, sv, sw)),
                                     _stream())
        return su, sv, sw

    def adjoint(self, u, v, w, dsu, dsv, dsw, out=None):
        du, dv, dw = out if out is not None else (self.empty(), self.empty(), self.empty())
        _abi.advect_ensemble_adjoint(self.handle, *(self._ptrs(x) for x in
                                                    (u, v, w, dsu, dsv, dsw, du, dv, dw)), _stream())
        return du, dv, dw

    def kernel_name(self, adjoint=False):
        return _abi.advect_kernel_name(self.handle, adjoint)

    def autotune(self, enable=True):
        _abi.advect_autotune(self.handle, enable)

    def tuned_config(self, adjoint=False):
        return _abi.advect_tuned_config(self.handle, adjoint)

    def sync(self):
        _abi.advect_sync(self.handle, _stream())

    def close(self):
        if self.handle:
            _abi.advect_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
