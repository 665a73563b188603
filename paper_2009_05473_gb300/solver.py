"""Sliding Frank-Wolfe (Algorithm 1) and its boosted variant (Algorithm 2) on the GPU path.

Every voxel-sized computation runs in libsfw: the residual and the criterion
(Eq. 4), the grid certificate with its device argmax and the off-grid
certificate with its gradient (step 1), the Gram system of the LASSO (step 3)
and the loss/gradient of the sliding descent (step 4 / 2b).  The host keeps
only the small dense FP64 work the method prescribes: the non-negative LASSO on
the k x k Gram matrix, the BFGS curvature updates and the line searches.

Readings of what the paper leaves open (same as the library's design notes):
the domain box D (m_a in [0, n_a - 1], sigma in [0.75, 4], d in [1.25, 3],
w >= 0), the stopping test max eta <= 1 + tau (tau = 1e-3), pruning of weights
<= 1e-10 max w, projected BFGS with Armijo backtracking, Lawson-Hanson NNLS.
"""

from __future__ import annotations

import time
from typing import Callable, Dict, List, Tuple

import numpy as np
import torch

from . import AtomSet, Plan

SIGMA_RANGE = (0.75, 4.0)
D_RANGE = (1.25, 3.0)


# ----------------------------------------------------------------------------- host FP64 pieces

def nonneg_quadratic_min(G: np.ndarray, q: np.ndarray, tol: float = 1e-12,
                         max_iter: int = 500) -> np.ndarray:
    """Minimise 1/2 w^T G w - q^T w over w >= 0 (G symmetric positive definite).

    Active-set method (Lawson & Hanson): grow the free set by the coordinate with
    the most negative gradient, solve the equality-constrained problem on it, and
    step back to the boundary whenever a free coordinate would turn negative."""
    n = q.size
    w = np.zeros(n)
    free = np.zeros(n, dtype=bool)
    qs = max(1.0, float(np.abs(q).max(initial=0.0)))
    for _ in range(max_iter):
        neg_grad = q - G @ w
        enter = np.where(~free & (neg_grad > tol * qs), neg_grad, -np.inf)
        if not np.isfinite(enter.max(initial=-np.inf)):
            break
        free[int(np.argmax(enter))] = True
        while True:
            f = np.flatnonzero(free)
            z = np.zeros(n)
            z[f] = np.linalg.solve(G[np.ix_(f, f)], q[f])
            if (z[f] > 0).all():
                w = z
                break
            blocked = free & (z <= 0)
            t = np.min(w[blocked] / (w[blocked] - z[blocked]))
            w = w + t * (z - w)
            free = free & (w > 1e-300)
            w[~free] = 0.0
    return w


def box_bfgs(fg: Callable[[np.ndarray], Tuple[float, np.ndarray]], x0: np.ndarray,
             lo: np.ndarray, hi: np.ndarray, gtol: float, max_iter: int = 200,
             f_rel_noise: float = 1e-6) -> Tuple[np.ndarray, float, int]:
    """Minimise on a box: BFGS on the variables not held at a bound, backtracking
    along the projected path, inverse-Hessian reset when the direction fails.

    A trial step is accepted by the Armijo test or, when the objective changed by
    less than its rounding level (f_rel_noise |f|: the loss and the certificate are
    summed from FP32 device values), by the approximate Wolfe condition of Hager and
    Zhang (SIAM J. Optim. 16, 2005): the slope along the step at the trial point is at
    most 0.8 of the slope's magnitude at the start.  Near a minimiser the Armijo
    decrease falls below the FP32 resolution of the loss while the gradient still
    points the way, so without the second test the search stops early."""
    x = np.minimum(np.maximum(np.asarray(x0, np.float64), lo), hi)
    f, g = fg(x)
    Hi = np.eye(x.size)
    it = 0
    for it in range(1, max_iter + 1):
        proj = x - np.minimum(np.maximum(x - g, lo), hi)
        if np.abs(proj).max(initial=0.0) <= gtol:
            break
        held = ((x <= lo) & (g > 0)) | ((x >= hi) & (g < 0))
        d = -(Hi @ np.where(held, 0.0, g))
        d[held] = 0.0
        if float(d @ g) >= 0.0:
            Hi = np.eye(x.size)
            d = np.where(held, 0.0, -g)
        step = 1.0
        for _ in range(50):
            xt = np.minimum(np.maximum(x + step * d, lo), hi)
            ft, gt = fg(xt)
            if np.isfinite(ft):
                gs = float(g @ (xt - x))
                if ft <= f + 1e-4 * gs:
                    break
                if gs < 0.0 and ft <= f + f_rel_noise * abs(f) and float(gt @ (xt - x)) <= -0.8 * gs:
                    break
            step *= 0.5
        else:
            break
        s, yv = xt - x, gt - g
        x, f, g = xt, ft, gt
        sy = float(s @ yv)
        if sy > 1e-12 * np.linalg.norm(s) * np.linalg.norm(yv):
            r = 1.0 / sy
            A = np.eye(x.size) - r * np.outer(s, yv)
            Hi = A @ Hi @ A.T + r * np.outer(s, s)
        if np.abs(s).max(initial=0.0) < 1e-13:
            break
    return x, f, it


# ----------------------------------------------------------------------------- the solver

class GPUSolver:
    """SFW / BSFW on one volume: y (device, FP32), PSF and certificate grid in `plan`."""

    def __init__(self, plan: Plan, y: torch.Tensor, lam: float, tau: float = 1e-3,
                 slide_gtol: float = 1e-6, ascent_gtol: float = 1e-7, topk: int = 0):
        self.plan, self.y, self.lam, self.tau = plan, y, float(lam), tau
        self.slide_gtol, self.ascent_gtol, self.topk = slide_gtol, ascent_gtol, topk
        n = plan.n
        self.lo1 = np.array([0.0, 0.0, 0.0, SIGMA_RANGE[0], D_RANGE[0]])
        self.hi1 = np.array([n[0] - 1.0, n[1] - 1.0, n[2] - 1.0, SIGMA_RANGE[1], D_RANGE[1]])
        self.stats = {"certificate": 0, "eta_points": 0, "slide_evals": 0, "gram": 0}
        # wall time of each kind of library call, from its launch until its results are on the
        # host (device work, launch overhead, atom uploads); the rest of a solve is host code
        self.call_seconds = {"certificate": 0.0, "eta_points": 0.0, "slide": 0.0, "gram": 0.0}

    def _timed(self, what: str, fn):
        t = time.perf_counter()
        out = fn()
        self.call_seconds[what] += time.perf_counter() - t
        return out

    # -- device calls --------------------------------------------------------------------
    def _atoms(self, thetas: np.ndarray, w: np.ndarray) -> AtomSet:
        return AtomSet.from_numpy(thetas[:, :3], thetas[:, 3], thetas[:, 4], w)

    def residual(self, thetas, w) -> torch.Tensor:
        if w.size == 0:
            return self.y
        _, _, r = self.plan.slide_loss_grad(self.y, self._atoms(thetas, w), self.lam,
                                            want_residual=True, want_grad=False)
        return r

    def criterion(self, thetas, w) -> float:
        if w.size == 0:
            return 0.5 * float((self.y.double() ** 2).sum().item())
        loss, _, _ = self.plan.slide_loss_grad(self.y, self._atoms(thetas, w), self.lam, want_grad=False)
        return float(loss.item())

    # -- step 1 --------------------------------------------------------------------------
    def _grid_argmax(self, thetas, w):
        r = self.residual(thetas, w)
        out = self.plan.certificate(r, self.lam, want_max=False)
        return r, int(out["best_idx"].item())

    def certificate_max(self, thetas, w):
        self.stats["certificate"] += 1
        if self.topk:
            def call():
                r = self.residual(thetas, w)
                return r, self.plan.certificate_topk(r, self.lam, self.topk)["best_theta"].double().cpu().numpy()
            r, theta0 = self._timed("certificate", call)
        else:
            r, flat = self._timed("certificate", lambda: self._grid_argmax(thetas, w))
            if flat < 0:
                raise FloatingPointError("certificate holds a NaN")
            k, lin = divmod(flat, self.plan.V)
            theta0 = np.concatenate([np.array(np.unravel_index(lin, self.plan.n), dtype=np.float64),
                                     self.plan.kernels[k]])

        def neg_eta(th):
            self.stats["eta_points"] += 1

            def call():
                e, g = self.plan.eta_points(r, self.lam, th[None, :])
                return -float(e.item()), -g[0].cpu().numpy()
            return self._timed("eta_points", call)

        th, f, _ = box_bfgs(neg_eta, theta0, self.lo1, self.hi1, gtol=self.ascent_gtol)
        return th, -f, theta0

    # -- step 3 --------------------------------------------------------------------------
    def lasso(self, thetas) -> np.ndarray:
        self.stats["gram"] += 1

        def call():
            G, c = self.plan.gram(self._atoms(thetas, np.ones(thetas.shape[0])), self.y)
            return G.cpu().numpy(), c.cpu().numpy()
        G, c = self._timed("gram", call)
        return nonneg_quadratic_min(G, c - self.lam)

    # -- step 4 / 2b ---------------------------------------------------------------------
    def slide(self, thetas, w, max_iter=300):
        k = w.size
        lo = np.concatenate([np.tile(self.lo1[:3], k), np.full(k, self.lo1[3]), np.full(k, self.lo1[4]), np.zeros(k)])
        hi = np.concatenate([np.tile(self.hi1[:3], k), np.full(k, self.hi1[3]), np.full(k, self.hi1[4]),
                             np.full(k, np.inf)])

        def fg(x):
            self.stats["slide_evals"] += 1
            th, ww = _unpack(x)

            def call():
                loss, grad, _ = self.plan.slide_loss_grad(self.y, self._atoms(th, ww), self.lam)
                return float(loss.item()), grad.cpu().numpy()
            return self._timed("slide", call)

        x, _, _ = box_bfgs(fg, _pack(thetas, w), lo, hi, gtol=self.slide_gtol, max_iter=max_iter)
        return _unpack(x)

    # -- Algorithms 1 and 2 ---------------------------------------------------------------
    def run(self, boosted: bool, max_iter: int = 50, log=None, thetas0=None, w0=None) -> Dict:
        thetas = np.zeros((0, 5)) if thetas0 is None else np.array(thetas0, np.float64).reshape(-1, 5)
        w = np.zeros(0) if w0 is None else np.array(w0, np.float64).ravel()
        if w.size:
            # a warm start: re-fit the given atoms' weights and positions at this lambda
            w = self.lasso(thetas)
            thetas, w = _prune(thetas, w)
            if w.size:
                thetas, w = self.slide(thetas, w)
                thetas, w = _prune(thetas, w)
        hist: List[Dict] = []
        t0 = time.perf_counter()
        for it in range(max_iter):
            th_new, eta_max, seed = self.certificate_max(thetas, w)
            rec = {"iter": it, "eta_max": eta_max, "seed": seed.tolist()}
            if eta_max > 1.0 + self.tau:
                thetas = np.vstack([thetas, th_new[None, :]])
                w = self.lasso(thetas)
                if not boosted:
                    thetas, w = self.slide(thetas, w)
                thetas, w = _prune(thetas, w)
                rec["n_atoms"] = int(w.size)
                hist.append(rec)
                if log:
                    log(rec)
                continue
            if boosted and w.size:
                thetas, w = self.slide(thetas, w)
                thetas, w = _prune(thetas, w)
            rec["n_atoms"] = int(w.size)
            hist.append(rec)
            if log:
                log(rec)
            break
        torch.cuda.synchronize()
        seconds = time.perf_counter() - t0
        stats = dict(self.stats)
        stats["call_seconds"] = dict(self.call_seconds)
        stats["host_seconds"] = seconds - sum(self.call_seconds.values())
        return {"thetas": thetas, "w": w, "C": self.criterion(thetas, w), "history": hist,
                "seconds": seconds, "stats": stats}


def _pack(thetas, w):
    return np.concatenate([thetas[:, :3].ravel(), thetas[:, 3], thetas[:, 4], w])


def _unpack(x):
    k = x.size // 6
    th = np.concatenate([x[:3 * k].reshape(k, 3), x[3 * k:4 * k, None], x[4 * k:5 * k, None]], 1)
    return th, x[5 * k:].copy()


def _prune(thetas, w):
    if w.size == 0:
        return thetas, w
    keep = w > 1e-10 * w.max()
    return thetas[keep], w[keep]


def lambda_max(plan: Plan, y: torch.Tensor) -> float:
    """Smallest lambda at which the empty measure passes the stopping test: the maximum of
    the correlation <Phi G(theta, 1), y> over the domain (the certificate of Eq. 5 at
    lambda = 1 with residual y), by step 1 of Algorithm 1 (grid argmax, then local ascent)."""
    _, eta, _ = GPUSolver(plan, y, 1.0).certificate_max(np.zeros((0, 5)), np.zeros(0))
    return float(eta)


def lambda_path(plan: Plan, y: torch.Tensor, fractions=(0.5, 0.2, 0.1, 0.05), boosted: bool = True,
                **kw) -> List[Dict]:
    """Solutions along decreasing lambda = f * lambda_max (f in fractions, decreasing), each
    solve warm-started from the previous one's atoms.  lambda only rescales the certificate
    (Eq. 5), so the certificate maximum of y fixes the scale of the whole path; fractions
    above 1 + tau give the empty measure."""
    lmax = lambda_max(plan, y)
    thetas, w = None, None
    path = []
    for f in sorted(fractions, reverse=True):
        lam = f * lmax
        out = GPUSolver(plan, y, lam, **kw).run(boosted=boosted, thetas0=thetas, w0=w)
        thetas, w = out["thetas"], out["w"]
        out["lambda"], out["fraction"] = lam, f
        path.append(out)
    return path


def sfw(plan: Plan, y: torch.Tensor, lam: float, **kw) -> Dict:
    """Sliding Frank-Wolfe (Algorithm 1) on the GPU path."""
    return GPUSolver(plan, y, lam, **kw).run(boosted=False)


def bsfw(plan: Plan, y: torch.Tensor, lam: float, **kw) -> Dict:
    """Boosted SFW (Algorithm 2) on the GPU path: one sliding descent, at the end."""
    return GPUSolver(plan, y, lam, **kw).run(boosted=True)
