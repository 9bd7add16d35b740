"""Torch-facing helpers over the C ABI: contexts, residual, VJP, autograd.

PyTorch provides device memory and streams only; every step of the volume
term runs in libsfhad's kernels.
"""
from __future__ import annotations

import torch

from . import _abi as A

NODES = {"gll": A.SFH_NODES_GLL, "gauss": A.SFH_NODES_GAUSS}
FLUX = {"burgers": A.SFH_FLUX_BURGERS, "euler": A.SFH_FLUX_EULER_RANOCHA,
        "euler_chandrashekar": A.SFH_FLUX_EULER_CHANDRASHEKAR}
BASIS = {"legendre": A.SFH_BASIS_LEGENDRE, "lagrange_gll": A.SFH_BASIS_LAGRANGE_GLL,
         "lagrange_gauss": A.SFH_BASIS_LAGRANGE_GAUSS}
PREC = {"fp64": A.SFH_FP64, "fp32k": A.SFH_FP32_KAHAN, "fp32mix": A.SFH_FP32_MIXED}
PREC_DTYPE = {A.SFH_FP64: torch.float64, A.SFH_FP32_KAHAN: torch.float32, A.SFH_FP32_MIXED: torch.float32}


def _enum(table, v):
    return table[v] if isinstance(v, str) else int(v)


class Context:
    """One element type: dimension d, degree p, node set, flux (owns an sfh_ctx)."""

    def __init__(self, d: int, p: int, nodes="gll", flux="euler"):
        self.d, self.p = d, p
        self.nodes = _enum(NODES, nodes)
        self.flux = _enum(FLUX, flux)
        self.nvar = 1 if self.flux == A.SFH_FLUX_BURGERS else d + 2
        self.n_nodes = (p + 1) ** d
        self.handle = A.sfh_create(d, p, self.nodes, self.nvar, self.flux)

    def close(self):
        if getattr(self, "handle", None):
            A.sfh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, stream=None) -> int:
        s = stream if stream is not None else torch.cuda.current_stream()
        return A.sfh_check(self.handle, s.cuda_stream)

    def _shape_check(self, u: torch.Tensor, Ja: torch.Tensor, dtype):
        E = u.shape[0]
        if u.shape != (E, self.nvar, self.n_nodes):
            raise ValueError(f"u must be [n_elem, {self.nvar}, {self.n_nodes}], got {tuple(u.shape)}")
        if Ja.shape != (E, self.d, self.d, self.n_nodes):
            raise ValueError(f"Ja must be [n_elem, {self.d}, {self.d}, {self.n_nodes}], got {tuple(Ja.shape)}")
        if u.dtype != dtype or Ja.dtype != torch.float64:
            raise TypeError(f"u must be {dtype} and Ja float64")
        if not (u.is_cuda and Ja.is_cuda and u.is_contiguous() and Ja.is_contiguous()):
            raise ValueError("u and Ja must be contiguous CUDA tensors")

    def volume_residual(self, u: torch.Tensor, Ja: torch.Tensor, prec="fp64", out: torch.Tensor | None = None):
        """r = sum_m (Q_m o F_m) 1 on the current stream (new tensor unless `out`)."""
        pr = _enum(PREC, prec)
        self._shape_check(u, Ja, PREC_DTYPE[pr])
        r = torch.empty_like(u) if out is None else out
        A.sfh_volume_residual(self.handle, u.shape[0], u.data_ptr(), Ja.data_ptr(), r.data_ptr(), pr,
                              torch.cuda.current_stream(u.device).cuda_stream)
        return r

    def volume_residual_modal(self, u_hat: torch.Tensor, Ja: torch.Tensor, basis="legendre", prec="fp64",
                              out: torch.Tensor | None = None):
        """r_hat = V^T r_v(V u_hat) for coefficients u_hat in ``basis`` (the
        modal / uncollocated path), on the current stream."""
        pr, b = _enum(PREC, prec), _enum(BASIS, basis)
        self._shape_check(u_hat, Ja, PREC_DTYPE[pr])
        r = torch.empty_like(u_hat) if out is None else out
        A.sfh_volume_residual_modal(self.handle, b, u_hat.shape[0], u_hat.data_ptr(), Ja.data_ptr(), r.data_ptr(),
                                    pr, torch.cuda.current_stream(u_hat.device).cuda_stream)
        return r

    def surface_hadamard(self, u: torch.Tensor, u_face: torch.Tensor, nJ_face: torch.Tensor):
        """(r_vol, r_face) of the surface Hadamard product of every element's
        faces (FP64) on the current stream."""
        E, d = u.shape[0], self.d
        nf = (self.p + 1) ** (d - 1)
        if u.shape != (E, self.nvar, self.n_nodes) or u_face.shape != (E, 2 * d, self.nvar, nf) \
                or nJ_face.shape != (E, 2 * d, d, nf):
            raise ValueError("u [E, nvar, n^d], u_face [E, 2d, nvar, n^(d-1)], nJ_face [E, 2d, d, n^(d-1)]")
        for t in (u, u_face, nJ_face):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("inputs must be contiguous float64 CUDA tensors")
        r_vol, r_face = torch.empty_like(u), torch.empty_like(u_face)
        A.sfh_surface_hadamard(self.handle, E, u.data_ptr(), u_face.data_ptr(), nJ_face.data_ptr(), r_vol.data_ptr(),
                               r_face.data_ptr(), torch.cuda.current_stream(u.device).cuda_stream)
        return r_vol, r_face

    def vjp_modal(self, u_hat: torch.Tensor, Ja: torch.Tensor, lam_hat: torch.Tensor, basis="legendre",
                  out: torch.Tensor | None = None):
        """V^T (dr_v/du_v)^T V lambda_hat (FP64), the VJP of volume_residual_modal."""
        self._shape_check(u_hat, Ja, torch.float64)
        if (lam_hat.shape != u_hat.shape or lam_hat.dtype != torch.float64 or not lam_hat.is_contiguous()
                or not lam_hat.is_cuda):
            raise ValueError("lambda_hat must be a contiguous float64 CUDA tensor shaped like u_hat")
        g = torch.empty_like(u_hat) if out is None else out
        A.sfh_vjp_modal(self.handle, _enum(BASIS, basis), u_hat.shape[0], u_hat.data_ptr(), Ja.data_ptr(),
                        lam_hat.data_ptr(), g.data_ptr(), torch.cuda.current_stream(u_hat.device).cuda_stream)
        return g

    def vjp(self, u: torch.Tensor, Ja: torch.Tensor, lam: torch.Tensor, out: torch.Tensor | None = None):
        """(dr/du)^T lambda (FP64) on the current stream."""
        self._shape_check(u, Ja, torch.float64)
        if lam.shape != u.shape or lam.dtype != torch.float64 or not lam.is_contiguous() or not lam.is_cuda:
            raise ValueError("lambda must be a contiguous float64 CUDA tensor shaped like u")
        g = torch.empty_like(u) if out is None else out
        A.sfh_vjp(self.handle, u.shape[0], u.data_ptr(), Ja.data_ptr(), lam.data_ptr(), g.data_ptr(),
                  torch.cuda.current_stream(u.device).cuda_stream)
        return g

    def entropy_residual(self, u: torch.Tensor, Ja: torch.Tensor, r: torch.Tensor) -> torch.Tensor:
        """Per-element defect of the entropy identity (FP64, on the GPU) of a
        residual r of this volume term (float64 or float32) at the FP64 state u."""
        self._shape_check(u, Ja, torch.float64)
        if r.shape != u.shape or not r.is_contiguous() or not r.is_cuda or r.dtype not in (torch.float64, torch.float32):
            raise ValueError("r must be a contiguous float32/float64 CUDA tensor shaped like u")
        out = torch.empty(u.shape[0], dtype=torch.float64, device=u.device)
        A.sfh_entropy_residual(self.handle, u.shape[0], u.data_ptr(), Ja.data_ptr(), r.data_ptr(),
                               A.SFH_FP64 if r.dtype == torch.float64 else A.SFH_FP32_KAHAN, out.data_ptr(),
                               torch.cuda.current_stream(u.device).cuda_stream)
        return out

    def volume_residual_host(self, u, Ja, prec="fp64"):
        """Host-buffer entry point: u, Ja CPU tensors (pinned for full speed); returns r on the host."""
        pr = _enum(PREC, prec)
        if u.is_cuda or Ja.is_cuda:
            raise ValueError("host entry point takes CPU tensors")
        r = torch.empty_like(u, pin_memory=u.is_pinned())
        st = A.sfh_volume_residual_host(self.handle, u.shape[0], u.data_ptr(), Ja.data_ptr(), r.data_ptr(), pr)
        if st != A.SFH_OK:
            raise A.SfhError(st, "sfh_volume_residual_host", A.sfh_last_error())
        return r


class SFHVolume(torch.autograd.Function):
    """r = volume_residual(u; Ja) with the hand-written adjoint as backward.
    FP64 only; Ja receives no gradient (it is geometry, held fixed)."""

    @staticmethod
    def forward(ctx_, u, Ja, context: Context):
        u = u.contiguous()
        ctx_.save_for_backward(u, Ja)
        ctx_.context = context
        return context.volume_residual(u, Ja, "fp64")

    @staticmethod
    def backward(ctx_, grad_r):
        u, Ja = ctx_.saved_tensors
        g = ctx_.context.vjp(u, Ja, grad_r.contiguous())
        return g, None, None


def volume(u: torch.Tensor, Ja: torch.Tensor, context: Context) -> torch.Tensor:
    """Differentiable FP64 volume residual (autograd through sfh_vjp)."""
    return SFHVolume.apply(u, Ja, context)


class SFHVolumeModal(torch.autograd.Function):
    """r_hat = volume_residual_modal(u_hat; Ja, basis) with the modal adjoint
    (sfh_vjp_modal) as backward.  FP64 only; Ja receives no gradient."""

    @staticmethod
    def forward(ctx_, u_hat, Ja, context: Context, basis):
        u_hat = u_hat.contiguous()
        ctx_.save_for_backward(u_hat, Ja)
        ctx_.context, ctx_.basis = context, basis
        return context.volume_residual_modal(u_hat, Ja, basis, "fp64")

    @staticmethod
    def backward(ctx_, grad_r):
        u_hat, Ja = ctx_.saved_tensors
        g = ctx_.context.vjp_modal(u_hat, Ja, grad_r.contiguous(), ctx_.basis)
        return g, None, None, None


def volume_modal(u_hat: torch.Tensor, Ja: torch.Tensor, context: Context, basis="legendre") -> torch.Tensor:
    """Differentiable FP64 modal volume residual (autograd through sfh_vjp_modal)."""
    return SFHVolumeModal.apply(u_hat, Ja, context, basis)
