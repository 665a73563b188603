"""GB300 hot path of the sliding Frank-Wolfe solver for 3D deconvolution (arXiv 2009.05473).

The compute lives in ``libsfw.so`` (hand-written CUDA for sm_103a, C ABI in
``include/sfw.h``).  This package marshals torch device tensors into those
calls; PyTorch only provides device memory and streams.  There is no CPU
path: without the built library every call raises.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

from . import _abi
from ._abi import (SfwError, sfw_argmax, sfw_certificate_grid, sfw_certificate_topk,  # noqa: F401
                   sfw_eta_points, sfw_forward, sfw_gram,
                   sfw_launch_count, sfw_plan_create, sfw_plan_destroy, sfw_plan_query,
                   sfw_plan_check, sfw_autotune, sfw_slide_loss_grad, sfw_step, sfw_step_topk, sfw_version)

__all__ = ["Plan", "AtomSet", "Batch", "argmax", "launch_count", "SfwError", "build_library"]


def build_library(force: bool = False) -> str:
    from .build import build
    return build(force=force)


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _f32(x, device) -> "torch.Tensor":
    torch = _torch()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device=device).contiguous()


@dataclass
class AtomSet:
    """Device atom set (FP32 structure of arrays): m (N, 3), sigma, d, w (N)."""

    m: "torch.Tensor"
    sigma: "torch.Tensor"
    d: "torch.Tensor"
    w: "torch.Tensor"

    @property
    def N(self) -> int:
        return int(self.w.shape[0])

    @staticmethod
    def from_numpy(m, sigma, d, w, device="cuda") -> "AtomSet":
        return AtomSet(_f32(np.reshape(m, (-1, 3)), device), _f32(sigma, device), _f32(d, device),
                       _f32(w, device))

    @staticmethod
    def from_params(x, device="cuda") -> "AtomSet":
        """From a 6N vector in gradient order [m (N x 3) | sigma | d | w]."""
        torch = _torch()
        x = torch.as_tensor(x, device=device).to(torch.float32)
        N = x.numel() // 6
        return AtomSet(x[:3 * N].reshape(N, 3).contiguous(), x[3 * N:4 * N].contiguous(),
                       x[4 * N:5 * N].contiguous(), x[5 * N:].contiguous())

    def abi(self) -> _abi.Atoms:
        for t in (self.m, self.sigma, self.d, self.w):
            if not (t.is_cuda and t.dtype == _torch().float32 and t.is_contiguous()):
                raise ValueError("atom arrays must be contiguous float32 CUDA tensors")
        return _abi.Atoms(self.N, _ptr(self.m), _ptr(self.sigma), _ptr(self.d), _ptr(self.w))


class Plan:
    """A geometry (grid n, PSF half-widths R, PSF H) plus a certificate grid of
    (sigma, d) kernels; owns the PSF spectrum, the kernel-family table and the
    device workspace (libsfw ``sfw_plan``)."""

    def __init__(self, n: Sequence[int], R: Sequence[int], psf, sigmas: Sequence[float] = (),
                 ds: Sequence[float] = (), precision: str = "fp32", eps: float = 0.0,
                 device: Optional[int] = None, route: str = "fft"):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2009_05473_gb300 needs a CUDA GPU (no CPU path)")
        if device is not None:
            torch.cuda.set_device(device)
        self.n = tuple(int(v) for v in n)
        self.R = tuple(int(v) for v in R)
        psf = np.ascontiguousarray(psf, dtype=np.float32)
        sig = np.ascontiguousarray(sigmas, dtype=np.float32)
        dd = np.ascontiguousarray(ds, dtype=np.float32)
        self.kernels = [(float(s), float(x)) for s in sig for x in dd]
        desc = _abi.PlanDesc()
        desc.n[:] = list(self.n)
        desc.R[:] = list(self.R)
        fp = ctypes.POINTER(ctypes.c_float)
        desc.psf = psf.ctypes.data_as(fp)
        desc.n_sigma = int(sig.size)
        desc.n_d = int(dd.size)
        desc.sigmas = sig.ctypes.data_as(fp) if sig.size else ctypes.cast(None, fp)
        desc.ds = dd.ctypes.data_as(fp) if dd.size else ctypes.cast(None, fp)
        desc.precision = {"fp32": _abi.SFW_PREC_FP32, "bf16": _abi.SFW_PREC_BF16}[precision]
        desc.eps = float(eps)
        desc.route = {"auto": _abi.SFW_ROUTE_AUTO, "fft": _abi.SFW_ROUTE_FFT,
                      "direct": _abi.SFW_ROUTE_DIRECT}[route]
        self._keep = (psf, sig, dd)
        self.handle = sfw_plan_create(desc)
        self._query()
        self.K = self.info["K"]
        self.V = int(np.prod(self.n))
        self.precision = precision
        self.route = route

    def _query(self):
        info = sfw_plan_query(self.handle)
        names = {_abi.SFW_ROUTE_FFT: "fft", _abi.SFW_ROUTE_DIRECT: "direct", 0: None}
        self.info = {"E": tuple(info.E), "P_conv": tuple(info.P_conv), "P_cert": tuple(info.P_cert),
                     "K": info.K, "real_table": bool(info.real_table),
                     "table_bytes": int(info.table_bytes), "workspace_bytes": int(info.workspace_bytes),
                     "route_blur": names[info.route_blur], "route_cert": names[info.route_cert],
                     "tensor_cores": bool(info.tensor_cores)}

    def autotune(self, cache_path: Optional[str] = None, stream=None) -> dict:
        """Engine choice by timing (libsfw ``sfw_autotune``): FFT or DIRECT per operation for a
        route="auto" plan, tensor cores or not for the axis-0 stage of a bf16 plan; returns the
        choices in use."""
        sfw_autotune(self.handle, cache_path, _stream_ptr(stream))
        self._query()
        return {"blur": self.info["route_blur"], "cert": self.info["route_cert"],
                "tensor_cores": self.info["tensor_cores"]}

    def close(self):
        if getattr(self, "handle", None):
            sfw_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the hot path ------------------------------------------------------------------
    def forward(self, atoms: AtomSet, out=None, stream=None):
        """Phi mu on the grid (Eq. 3 without noise)."""
        torch = _torch()
        y = out if out is not None else torch.empty(self.n, dtype=torch.float32, device="cuda")
        sfw_forward(self.handle, atoms.abi(), _ptr(y), _stream_ptr(stream))
        return y

    def certificate(self, residual, lam: float, want_eta: bool = False, want_max: bool = True,
                    stream=None, out=None):
        """Grid certificate (Eq. 5): dict with max (n), argk (n), best_val, best_idx, eta (K, n)."""
        torch = _torch()
        out = out or {}
        eta = out.get("eta")
        if want_eta and eta is None:
            eta = torch.empty((self.K,) + self.n, dtype=torch.float32, device="cuda")
        mx = out.get("max")
        ak = out.get("argk")
        if want_max and mx is None:
            mx = torch.empty(self.n, dtype=torch.float32, device="cuda")
            ak = torch.empty(self.n, dtype=torch.int32, device="cuda")
        bv = out.get("best_val")
        bi = out.get("best_idx")
        if bv is None:
            bv = torch.empty(1, dtype=torch.float32, device="cuda")
            bi = torch.empty(1, dtype=torch.int64, device="cuda")
        sfw_certificate_grid(self.handle, _ptr(residual), lam, _ptr(eta) if want_eta else 0,
                             _ptr(mx) if want_max else 0, _ptr(ak) if want_max else 0, _ptr(bv),
                             _ptr(bi), _stream_ptr(stream))
        return {"eta": eta if want_eta else None, "max": mx if want_max else None,
                "argk": ak if want_max else None, "best_val": bv, "best_idx": bi}

    def certificate_topk(self, residual, lam: float, topk: int = 64, stream=None):
        """Grid certificate, its topk voxels and their FP32 re-scores: dict with theta
        (topk, 5), grid (topk), eta (topk, FP64 output of FP32 sums), best_theta (5), best_eta."""
        torch = _torch()
        th = torch.empty((topk, 5), dtype=torch.float32, device="cuda")
        gv = torch.empty(topk, dtype=torch.float32, device="cuda")
        ev = torch.empty(topk, dtype=torch.float64, device="cuda")
        bt = torch.empty(5, dtype=torch.float32, device="cuda")
        be = torch.empty(1, dtype=torch.float64, device="cuda")
        sfw_certificate_topk(self.handle, _ptr(residual), lam, topk, _ptr(th), _ptr(gv), _ptr(ev),
                             _ptr(bt), _ptr(be), _stream_ptr(stream))
        return {"theta": th, "grid": gv, "eta": ev, "best_theta": bt, "best_eta": be}

    def gram(self, atoms: AtomSet, y, stream=None):
        """(G, c): G[i][j] = <Phi G(theta_i,1), Phi G(theta_j,1)>, c[i] = <Phi G(theta_i,1), y>."""
        torch = _torch()
        G = torch.empty((atoms.N, atoms.N), dtype=torch.float64, device="cuda")
        c = torch.empty(atoms.N, dtype=torch.float64, device="cuda")
        sfw_gram(self.handle, atoms.abi(), _ptr(y), _ptr(G), _ptr(c), _stream_ptr(stream))
        return G, c

    def eta_points(self, residual, lam: float, theta, with_grad: bool = True, stream=None):
        """eta (and d eta / d theta) at rows theta = (m0, m1, m2, sigma, d), FP32 sums."""
        torch = _torch()
        th = torch.as_tensor(theta, dtype=torch.float32, device="cuda").reshape(-1, 5).contiguous()
        P = th.shape[0]
        eta = torch.empty(P, dtype=torch.float64, device="cuda")
        grad = torch.empty((P, 5), dtype=torch.float64, device="cuda") if with_grad else None
        sfw_eta_points(self.handle, _ptr(residual), lam, P, _ptr(th), _ptr(eta), _ptr(grad),
                       _stream_ptr(stream))
        return (eta, grad) if with_grad else eta

    def slide_loss_grad(self, y, atoms: AtomSet, lam: float, want_residual: bool = False,
                        stream=None, out=None, want_grad: bool = True):
        """(loss (1 double), grad (6N doubles) or None, residual or None) of the sliding step."""
        torch = _torch()
        out = out or {}
        loss = out.get("loss")
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device="cuda")
        grad = out.get("grad") if want_grad else None
        if want_grad and (grad is None or grad.numel() != 6 * atoms.N):
            grad = torch.empty(6 * atoms.N, dtype=torch.float64, device="cuda")
        r = out.get("residual")
        if want_residual and r is None:
            r = torch.empty(self.n, dtype=torch.float32, device="cuda")
        sfw_slide_loss_grad(self.handle, _ptr(y), atoms.abi(), lam, _ptr(loss), _ptr(grad),
                            _ptr(r) if want_residual else 0, _stream_ptr(stream))
        return loss, grad, (r if want_residual else None)

    def check(self):
        """Raise SfwError (SFW_ERR_TIMEOUT) if a bounded device wait of this plan's kernels ran
        out since the last check (synchronises the device)."""
        sfw_plan_check(self.handle)

    def step(self, y, atoms: AtomSet, lam: float, aux_stream=None, stream=None, out=None,
             want_grad: bool = True):
        """One SFW iteration's device work (libsfw ``sfw_step``): the sliding loss, its
        gradient and the residual, and the grid certificate maximum of that residual.  With
        ``aux_stream`` (a torch.cuda.Stream) the certificate overlaps the back-projection.
        Returns dict(loss, grad, residual, best_val, best_idx)."""
        torch = _torch()
        out = {} if out is None else out
        if out.get("loss") is None:
            out["loss"] = torch.empty(1, dtype=torch.float64, device="cuda")
        if want_grad and (out.get("grad") is None or out["grad"].numel() != 6 * atoms.N):
            out["grad"] = torch.empty(6 * atoms.N, dtype=torch.float64, device="cuda")
        if out.get("residual") is None:
            out["residual"] = torch.empty(self.n, dtype=torch.float32, device="cuda")
        if out.get("best_val") is None:
            out["best_val"] = torch.empty(1, dtype=torch.float32, device="cuda")
        if out.get("best_idx") is None:
            out["best_idx"] = torch.empty(1, dtype=torch.int64, device="cuda")
        sfw_step(self.handle, _ptr(y), atoms.abi(), lam, _ptr(out["loss"]),
                 _ptr(out["grad"]) if want_grad else 0, _ptr(out["residual"]), _ptr(out["best_val"]),
                 _ptr(out["best_idx"]), _stream_ptr(stream),
                 int(aux_stream.cuda_stream) if aux_stream is not None else 0)
        return out

    def step_topk(self, y, atoms: AtomSet, lam: float, topk: int = 64, aux_stream=None, stream=None,
                  out=None):
        """The same iteration with the precision configuration's seed (libsfw ``sfw_step_topk``):
        the sliding loss, gradient and residual, and the grid certificate's topk voxels
        re-scored in FP32, one back-projection serving both.  With ``aux_stream`` the
        certificate overlaps the back-projection and the adjoint sums.  Returns dict(loss,
        grad, residual, theta, grid, eta, best_theta, best_eta)."""
        torch = _torch()
        out = {} if out is None else out
        shapes = {"loss": ((1,), torch.float64), "grad": ((6 * atoms.N,), torch.float64),
                  "residual": (tuple(self.n), torch.float32), "theta": ((topk, 5), torch.float32),
                  "grid": ((topk,), torch.float32), "eta": ((topk,), torch.float64),
                  "best_theta": ((5,), torch.float32), "best_eta": ((1,), torch.float64)}
        for k, (shape, dt) in shapes.items():
            if out.get(k) is None or tuple(out[k].shape) != shape:
                out[k] = torch.empty(shape, dtype=dt, device="cuda")
        sfw_step_topk(self.handle, _ptr(y), atoms.abi(), lam, _ptr(out["loss"]), _ptr(out["grad"]),
                      _ptr(out["residual"]), topk, _ptr(out["theta"]), _ptr(out["grid"]), _ptr(out["eta"]),
                      _ptr(out["best_theta"]), _ptr(out["best_eta"]), _stream_ptr(stream),
                      int(aux_stream.cuda_stream) if aux_stream is not None else 0)
        return out


class Batch:
    """Independent volumes (each with its own Plan) stepped together: one SFW iteration's hot
    path per volume (loss, gradient, residual, grid argmax) through grouped persistent launches
    (libsfw ``sfw_batch``).  The input tensors (y and the atoms) are read in place at every
    step: update them with in-place copies.  Outputs: loss (count), best_val, best_idx (count),
    residual[v], grad[v]."""

    def __init__(self, plans: Sequence[Plan], ys, atoms: Sequence[AtomSet], lambdas: Sequence[float]):
        torch = _torch()
        self.plans = list(plans)
        self.ys = list(ys)
        self.atoms = list(atoms)
        count = len(self.plans)
        self.loss = torch.empty(count, dtype=torch.float64, device="cuda")
        self.best_val = torch.empty(count, dtype=torch.float32, device="cuda")
        self.best_idx = torch.empty(count, dtype=torch.int64, device="cuda")
        self.residual = [torch.empty(p.n, dtype=torch.float32, device="cuda") for p in self.plans]
        self.grad = [torch.empty(6 * a.N, dtype=torch.float64, device="cuda") for a in self.atoms]
        vols = []
        for v in range(count):
            a = self.atoms[v]
            a.abi()  # validates the atom tensors
            if not (self.ys[v].is_cuda and self.ys[v].dtype == torch.float32 and self.ys[v].is_contiguous()):
                raise ValueError("y must be a contiguous float32 CUDA tensor")
            vols.append(_abi.BatchVolume(a.N, _ptr(self.ys[v]), _ptr(a.m), _ptr(a.sigma), _ptr(a.d),
                                         _ptr(a.w), _ptr(self.residual[v]), _ptr(self.grad[v]),
                                         _ptr(self.loss[v:v + 1]), _ptr(self.best_val[v:v + 1]),
                                         _ptr(self.best_idx[v:v + 1])))
        self.handle = _abi.sfw_batch_create([p.handle for p in self.plans], vols, lambdas)
        self.launches_per_step = _abi.sfw_batch_query(self.handle)

    def step(self, stream=None):
        _abi.sfw_batch_step(self.handle, _stream_ptr(stream))

    def autotune(self, cache_path: Optional[str] = None, stream=None):
        """Pick the persistent grid of every grouped launch by timing (cached in cache_path)."""
        _abi.sfw_batch_autotune(self.handle, cache_path, _stream_ptr(stream))

    def close(self):
        if getattr(self, "handle", None):
            _abi.sfw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def argmax(values, topk: int = 1, stream=None) -> Tuple["torch.Tensor", "torch.Tensor"]:
    """(values, flat indices) of the topk largest entries, ties to the lowest index."""
    torch = _torch()
    v = values.contiguous()
    vals = torch.empty(topk, dtype=torch.float32, device="cuda")
    idx = torch.empty(topk, dtype=torch.int64, device="cuda")
    sfw_argmax(_ptr(v), v.numel(), topk, _ptr(vals), _ptr(idx), _stream_ptr(stream))
    return vals, idx


def launch_count() -> int:
    """Kernels launched by libsfw in this process."""
    return sfw_launch_count()
