"""FP64 CPU oracle for the sliding Frank-Wolfe (SFW) solver of arXiv 2009.05473.

TEST INFRASTRUCTURE ONLY: only tests, the package smoke check and the
benchmark's CPU-baseline leg import this module.  The product library never
does, and this module never imports the product package.

The voxel sums (render, blur, back-projection, certificate at given points and
the analytic gradient) are the plain definitions in ``sfw_oracle.c``, loaded
with ctypes.  This file adds, in numpy, float64:

  * the criterion C of Eq. 4 and its gradient (render -> blur -> residual ->
    back-projection -> per-atom sums);
  * Fourier-domain variants of the blur, back-projection and grid certificate
    (Section 2 states that convolutions are made in the Fourier domain).  A
    library FFT (scipy.fft, all host threads) is one step; the result equals the direct definition up to
    rounding.  They are pinned against the direct sums in the tests and only
    make the larger cases affordable;
  * the certificate on the grid (positions x sigma-list x d-list) and its
    argmax (ties to the lowest flat index k*V + lin(m));
  * the non-negative LASSO of step 3 (Lawson-Hanson active set on the Gram
    form);
  * projected BFGS for the local ascent of step 1 and the local descent of
    step 4 (Algorithm 1) / step 2b (Algorithm 2);
  * SFW (Algorithm 1) and BSFW (Algorithm 2).

Readings of points the paper leaves open (each listed in the design notes):
domain box D = {m_a in [0, n_a-1], sigma in [0.75, 4], d in [1.25, 3], w >= 0};
the stopping test is max eta <= 1 + tau with tau = 1e-3; the prune threshold
is w <= 1e-10 max w; lambda = 0.05 max over the grid of Phi^T y.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np
import scipy.fft as sfft

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsfw_oracle.so")

SIGMA_BOUNDS = (0.75, 4.0)
D_BOUNDS = (1.25, 3.0)
# stopping test of Algorithms 1 and 2: stop once max eta <= 1 + TAU (the paper writes "> 1"
# to continue and "< 1" to stop; the margin covers the rounding spread of a converged slide)
TAU = 1e-3
PRUNE_REL = 1e-10

__all__ = [
    "build_oracle", "lib", "num_threads", "render", "forward_conv", "backproject", "eta_points",
    "atom_grad", "argmax", "forward", "forward_fft", "backproject_fft", "observe", "criterion",
    "loss_and_grad", "grid_thetas", "eta_grid", "eta_grid_fft", "grid_argmax", "lambda_rule", "nnls_gram",
    "lasso_weights", "atom_columns", "projected_bfgs", "sfw", "bsfw", "domain_bounds", "pack_params",
    "unpack_params", "SIGMA_BOUNDS", "D_BOUNDS", "TAU",
]


# ----------------------------------------------------------------------------- build / load

def build_oracle(force: bool = False) -> str:
    """Compile sfw_oracle.c (gcc -O2 -fopenmp) into oracle/_build; return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_render.argtypes = [_ip, _ip, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        L.oracle_forward_conv.argtypes = [_ip, _ip, _dp, _dp, _dp]
        L.oracle_backproject.argtypes = [_ip, _ip, _dp, _dp, _dp]
        L.oracle_eta_points.argtypes = [_ip, _ip, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
        L.oracle_atom_grad.argtypes = [_ip, _ip, ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
                                       ctypes.c_double, _dp]
        L.oracle_argmax.argtypes = [_dp, ctypes.c_int64]
        L.oracle_argmax.restype = ctypes.c_int64
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i3(v) -> ctypes.Array:
    return (ctypes.c_int * 3)(*[int(x) for x in v])


def ext_shape(n, R) -> Tuple[int, int, int]:
    return tuple(int(a) + 2 * int(r) for a, r in zip(n, R))


# ----------------------------------------------------------------------------- direct sums

def render(n, R, m, sigma, d, w) -> np.ndarray:
    """Sum of the atoms of Eq. 2 sampled on the extended grid E (untruncated)."""
    m, sigma, d, w = _c(np.reshape(m, (-1, 3))), _c(sigma), _c(d), _c(w)
    f = np.empty(ext_shape(n, R))
    lib().oracle_render(_i3(n), _i3(R), int(w.shape[0]), _p(m), _p(sigma), _p(d), _p(w), _p(f))
    return f


def forward_conv(n, R, psf, f) -> np.ndarray:
    """Eq. 3 restricted to the grid: y(s) = sum_t H(s - t) f(t) (brute force)."""
    psf, f = _c(psf), _c(f)
    assert f.shape == ext_shape(n, R) and psf.shape == tuple(2 * r + 1 for r in R)
    y = np.empty(tuple(n))
    lib().oracle_forward_conv(_i3(n), _i3(R), _p(psf), _p(f), _p(y))
    return y


def backproject(n, R, psf, r) -> np.ndarray:
    """Transpose of forward_conv: b(t) = sum_s H(s - t) r(s) on E (brute force)."""
    psf, r = _c(psf), _c(r)
    assert r.shape == tuple(n)
    b = np.empty(ext_shape(n, R))
    lib().oracle_backproject(_i3(n), _i3(R), _p(psf), _p(r), _p(b))
    return b


def eta_points(n, R, b, lam, theta, with_grad=False):
    """Eq. 5 at arbitrary theta rows (m0, m1, m2, sigma, d): (1/lam) sum_t g_theta(t) b(t)."""
    b = _c(b)
    theta = _c(np.reshape(theta, (-1, 5)))
    P = theta.shape[0]
    eta = np.empty(P)
    grad = np.empty((P, 5)) if with_grad else None
    lib().oracle_eta_points(_i3(n), _i3(R), _p(b), float(lam), P, _p(theta), _p(eta),
                            _p(grad) if with_grad else ctypes.cast(None, _dp))
    return (eta, grad) if with_grad else eta


def atom_grad(n, R, m, sigma, d, w, b, lam) -> np.ndarray:
    """Analytic dC/d(m, sigma, d, w) given b = backprojection of the residual (6N vector)."""
    m, sigma, d, w, b = _c(np.reshape(m, (-1, 3))), _c(sigma), _c(d), _c(w), _c(b)
    N = int(w.shape[0])
    g = np.empty(6 * N)
    lib().oracle_atom_grad(_i3(n), _i3(R), N, _p(m), _p(sigma), _p(d), _p(w), _p(b), float(lam),
                           _p(g))
    return g


def argmax(v) -> int:
    """Index of the maximum, ties to the lowest index, -1 if v holds a NaN."""
    v = _c(np.ravel(v))
    return int(lib().oracle_argmax(_p(v), int(v.size)))


# ----------------------------------------------------------------------------- Fourier variants

def _fft_shape(shape) -> Tuple[int, ...]:
    return tuple(int(s) for s in shape)


_WORKERS = os.cpu_count() or 1
_AX = (0, 1, 2)


def _rfftn(a, shape):
    return sfft.rfftn(a, shape, axes=_AX, workers=_WORKERS)


def _irfftn(a, shape):
    return sfft.irfftn(a, shape, axes=_AX, workers=_WORKERS)


def _wrapped_psf(psf, R, P) -> np.ndarray:
    """H(u), u in [-R, R], stored at u mod P (circular layout of the kernel)."""
    Hp = np.zeros(P)
    Hp[:psf.shape[0], :psf.shape[1], :psf.shape[2]] = psf
    return np.roll(Hp, shift=(-R[0], -R[1], -R[2]), axis=(0, 1, 2))


def forward_fft(n, R, psf, f) -> np.ndarray:
    """forward_conv through a zero-padded FFT of size E (linear, no wrap onto the grid)."""
    E = ext_shape(n, R)
    P = _fft_shape(E)
    Hp = _wrapped_psf(psf, R, P)
    out = _irfftn(_rfftn(f, P) * _rfftn(Hp, P), P)
    return out[R[0]:R[0] + n[0], R[1]:R[1] + n[1], R[2]:R[2] + n[2]].copy()


def backproject_fft(n, R, psf, r) -> np.ndarray:
    """backproject through FFT: correlation of the grid residual with H, on E."""
    E = ext_shape(n, R)
    P = _fft_shape(E)
    Hp = _wrapped_psf(psf, R, P)
    rE = np.zeros(P)
    rE[R[0]:R[0] + n[0], R[1]:R[1] + n[1], R[2]:R[2] + n[2]] = r
    return _irfftn(_rfftn(rE, P) * np.conj(_rfftn(Hp, P)), P)


def forward(n, R, psf, m, sigma, d, w, fft=False) -> np.ndarray:
    """Phi mu (Eq. 3 without noise), on the grid."""
    f = render(n, R, m, sigma, d, w)
    return forward_fft(n, R, psf, f) if fft else forward_conv(n, R, psf, f)


def observe(vol, fft=True) -> np.ndarray:
    """Noisy observation y = Phi mu* + noise_frac * max(Phi mu*) * z (Eq. 1), float64."""
    y0 = forward(vol.n, vol.R, vol.psf, vol.m, vol.sigma, vol.d, vol.w, fft=fft)
    return y0 + vol.noise_frac * float(y0.max()) * vol.noise


def criterion(n, R, psf, y, m, sigma, d, w, lam, fft=False) -> float:
    """C(y, mu, lambda) = 1/2 |y - Phi mu|^2 + lambda sum w (Eq. 4)."""
    r = y - forward(n, R, psf, m, sigma, d, w, fft=fft)
    return 0.5 * float(np.sum(r * r)) + lam * float(np.sum(w))


def loss_and_grad(n, R, psf, y, m, sigma, d, w, lam, fft=False):
    """(C, dC/dparams, residual); the gradient follows the analytic adjoint (Section 2)."""
    f = render(n, R, m, sigma, d, w)
    phi = forward_fft(n, R, psf, f) if fft else forward_conv(n, R, psf, f)
    r = y - phi
    C = 0.5 * float(np.sum(r * r)) + lam * float(np.sum(w))
    b = backproject_fft(n, R, psf, r) if fft else backproject(n, R, psf, r)
    return C, atom_grad(n, R, m, sigma, d, w, b, lam), r


# ----------------------------------------------------------------------------- grid certificate

def grid_thetas(n, kernels: Sequence[Tuple[float, float]]) -> np.ndarray:
    """All grid candidates in flat order k*V + lin(m): rows (m0, m1, m2, sigma_k, d_k)."""
    idx = np.indices(tuple(n)).reshape(3, -1).T.astype(np.float64)
    rows = []
    for s, dd in kernels:
        rows.append(np.concatenate([idx, np.full((idx.shape[0], 1), s), np.full((idx.shape[0], 1), dd)], 1))
    return np.concatenate(rows, 0)


def eta_grid(n, R, psf, r, lam, kernels, b=None) -> np.ndarray:
    """Certificate on the grid by the direct definition: (K, n0, n1, n2)."""
    if b is None:
        b = backproject(n, R, psf, r)
    eta = eta_points(n, R, b, lam, grid_thetas(n, kernels))
    return eta.reshape((len(kernels),) + tuple(n))


def atom_profile_window(half, sigma, d) -> np.ndarray:
    """g_{sigma,d}(j) = exp(-(1/2)(|j|/sigma)^d) on integer offsets |j_a| <= half_a."""
    ax = [np.arange(-h, h + 1, dtype=np.float64) for h in half]
    rho = np.sqrt(ax[0][:, None, None] ** 2 + ax[1][None, :, None] ** 2 + ax[2][None, None, :] ** 2)
    return np.exp(-0.5 * (rho / sigma) ** d)


def eta_grid_fft(n, R, psf, r, lam, kernels, b=None) -> np.ndarray:
    """Certificate on the grid through a library FFT: correlation of b (on E) with g_k."""
    if b is None:
        b = backproject_fft(n, R, psf, r)
    half = tuple(int(a) + int(rr) - 1 for a, rr in zip(n, R))      # |t - R - m| <= n + R - 1
    Q = tuple(2 * h + 1 for h in half)
    Bh = _rfftn(b, Q)
    out = np.empty((len(kernels),) + tuple(n))
    for k, (s, dd) in enumerate(kernels):
        g = atom_profile_window(half, s, dd)                      # g is even: correlation == conv
        c = _irfftn(Bh * _rfftn(g, Q), Q)                         # c[z + half] = sum_t b(t) g(z - t)
        out[k] = c[R[0] + half[0]:R[0] + half[0] + n[0], R[1] + half[1]:R[1] + half[1] + n[1],
                   R[2] + half[2]:R[2] + half[2] + n[2]] / lam
    return out


def grid_argmax(eta) -> Tuple[int, float]:
    """(flat index k*V + lin(m), value) of the certificate maximum, ties to the lowest index."""
    i = argmax(eta)
    if i < 0:
        raise FloatingPointError("certificate holds a NaN")
    return i, float(np.ravel(eta)[i])


def lambda_rule(n, R, psf, y, kernels, frac=0.05, fft=True) -> float:
    """lambda = frac * max over the certificate grid of Phi^T y (so the first max eta = 1/frac)."""
    eta = (eta_grid_fft if fft else eta_grid)(n, R, psf, y, 1.0, kernels)
    return frac * float(eta.max())


# ----------------------------------------------------------------------------- LASSO (step 3)

def nnls_gram(A: np.ndarray, q: np.ndarray, tol: float = 1e-12, max_outer: int = 1000) -> np.ndarray:
    """argmin_{w >= 0} 1/2 w^T A w - q^T w for SPD A (Lawson-Hanson active set, Gram form)."""
    A = np.asarray(A, np.float64)
    q = np.asarray(q, np.float64)
    n = q.shape[0]
    w = np.zeros(n)
    P = np.zeros(n, dtype=bool)
    scale = max(1.0, float(np.max(np.abs(q))) if n else 1.0)
    for _ in range(max_outer):
        dual = q - A @ w                       # minus the gradient
        cand = (~P) & (dual > tol * scale)
        if not cand.any():
            break
        j = int(np.argmax(np.where(cand, dual, -np.inf)))
        P[j] = True
        for _inner in range(10 * n + 10):
            z = np.zeros(n)
            idx = np.flatnonzero(P)
            z[idx] = np.linalg.solve(A[np.ix_(idx, idx)], q[idx])
            if np.all(z[idx] > 0):
                w = z
                break
            bad = P & (z <= 0)
            alpha = float(np.min(w[bad] / (w[bad] - z[bad])))
            w = w + alpha * (z - w)
            P &= w > tol * 1e-3 * max(1.0, float(np.max(np.abs(w))))
            w[~P] = 0.0
    return w


def atom_columns(n, R, psf, thetas, fft=False) -> np.ndarray:
    """a_i = Phi G(theta_i, 1) for each atom, as (k, V) rows."""
    cols = []
    for th in np.reshape(thetas, (-1, 5)):
        cols.append(forward(n, R, psf, th[None, :3], th[3:4], th[4:5], np.ones(1), fft=fft).ravel())
    return np.array(cols)


def lasso_weights(n, R, psf, y, thetas, lam, fft=False) -> np.ndarray:
    """Step 3: argmin_{w >= 0} C(y, mu_{w, theta}, lambda) at fixed theta."""
    Acol = atom_columns(n, R, psf, thetas, fft=fft)
    G = Acol @ Acol.T
    c = Acol @ np.ravel(y)
    return nnls_gram(G, c - lam)


# ----------------------------------------------------------------------------- projected BFGS

def projected_bfgs(fun: Callable[[np.ndarray], Tuple[float, np.ndarray]], x0, lo, hi,
                   gtol: float = 1e-6, max_iter: int = 200, c1: float = 1e-4):
    """Minimise fun on the box [lo, hi] by BFGS on the free variables, with an Armijo
    backtracking search along the projected path.  Returns (x, f, iterations)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    x = np.clip(np.asarray(x0, np.float64), lo, hi)
    f, g = fun(x)
    n = x.size
    Hinv = np.eye(n)
    it = 0
    for it in range(1, max_iter + 1):
        pg = x - np.clip(x - g, lo, hi)
        if np.max(np.abs(pg)) <= gtol:
            break
        active = ((x <= lo) & (g > 0)) | ((x >= hi) & (g < 0))
        free = ~active
        p = np.zeros(n)
        Hf = Hinv[np.ix_(free, free)]
        p[free] = -Hf @ g[free]
        if g @ p >= 0:
            Hinv = np.eye(n)
            p = np.where(free, -g, 0.0)
        alpha = 1.0
        accepted = False
        for _ in range(60):
            xn = np.clip(x + alpha * p, lo, hi)
            fn, gn = fun(xn)
            if np.isfinite(fn) and fn <= f + c1 * (g @ (xn - x)):
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            break
        s = xn - x
        yv = gn - g
        sy = float(s @ yv)
        x, f, g = xn, fn, gn
        if sy > 1e-12 * max(1.0, float(np.linalg.norm(s) * np.linalg.norm(yv))):
            rho = 1.0 / sy
            I = np.eye(n)
            V = I - rho * np.outer(s, yv)
            Hinv = V @ Hinv @ V.T + rho * np.outer(s, s)
        if np.max(np.abs(s)) < 1e-14:
            break
    return x, f, it


# ----------------------------------------------------------------------------- SFW / BSFW

def domain_bounds(n) -> Tuple[np.ndarray, np.ndarray]:
    """Per-atom box of D: (m0, m1, m2, sigma, d)."""
    lo = np.array([0.0, 0.0, 0.0, SIGMA_BOUNDS[0], D_BOUNDS[0]])
    hi = np.array([n[0] - 1.0, n[1] - 1.0, n[2] - 1.0, SIGMA_BOUNDS[1], D_BOUNDS[1]])
    return lo, hi


def pack_params(thetas: np.ndarray, w: np.ndarray) -> np.ndarray:
    """(k x 5 thetas, k weights) -> 6k vector in gradient order (m, sigma, d, w)."""
    th = np.reshape(thetas, (-1, 5))
    return np.concatenate([th[:, :3].ravel(), th[:, 3], th[:, 4], np.asarray(w, np.float64)])


def unpack_params(x: np.ndarray):
    k = x.size // 6
    m = x[:3 * k].reshape(k, 3)
    th = np.concatenate([m, x[3 * k:4 * k, None], x[4 * k:5 * k, None]], 1)
    return th, x[5 * k:6 * k].copy()


def _certificate_max(n, R, psf, y, thetas, w, lam, kernels, fft):
    """Step 1: grid maximum of eta, then a local ascent (projected BFGS on -eta)."""
    th = np.reshape(thetas, (-1, 5))
    if th.shape[0]:
        r = y - forward(n, R, psf, th[:, :3], th[:, 3], th[:, 4], w, fft=fft)
    else:
        r = np.array(y, dtype=np.float64, copy=True)
    b = backproject_fft(n, R, psf, r) if fft else backproject(n, R, psf, r)
    eta = (eta_grid_fft if fft else eta_grid)(n, R, psf, r, lam, kernels, b=b)
    flat, _val = grid_argmax(eta)
    V = int(np.prod(n))
    k, lin = divmod(flat, V)
    m0 = np.array(np.unravel_index(lin, tuple(n)), dtype=np.float64)
    theta0 = np.concatenate([m0, [kernels[k][0], kernels[k][1]]])
    lo, hi = domain_bounds(n)

    def neg_eta(x):
        e, g = eta_points(n, R, b, lam, x[None, :], with_grad=True)
        return -float(e[0]), -g[0]

    x, f, _ = projected_bfgs(neg_eta, theta0, lo, hi, gtol=1e-7, max_iter=200)
    return x, -f, flat


def _slide(n, R, psf, y, thetas, w, lam, fft, max_iter=300):
    """Local descent of C on all (m, sigma, d, w) of the current atoms (projected BFGS)."""
    k = np.reshape(thetas, (-1, 5)).shape[0]
    lo1, hi1 = domain_bounds(n)
    lo = np.concatenate([np.tile(lo1[:3], k), np.full(k, lo1[3]), np.full(k, lo1[4]), np.zeros(k)])
    hi = np.concatenate([np.tile(hi1[:3], k), np.full(k, hi1[3]), np.full(k, hi1[4]), np.full(k, np.inf)])

    def fun(x):
        th, ww = unpack_params(x)
        C, g, _ = loss_and_grad(n, R, psf, y, th[:, :3], th[:, 3], th[:, 4], ww, lam, fft=fft)
        return C, g

    x, f, _ = projected_bfgs(fun, pack_params(thetas, w), lo, hi, gtol=1e-7, max_iter=max_iter)
    return unpack_params(x)


def _prune(thetas, w):
    th = np.reshape(thetas, (-1, 5))
    if w.size == 0:
        return th, w
    keep = w > PRUNE_REL * max(float(np.max(w)), 0.0)
    return th[keep], w[keep]


def _run(n, R, psf, y, lam, kernels, boosted, fft, tau, max_iter, log):
    thetas = np.zeros((0, 5))
    w = np.zeros(0)
    history: List[Dict] = []
    for it in range(max_iter):
        theta_new, eta_max, flat = _certificate_max(n, R, psf, y, thetas, w, lam, kernels, fft)
        rec = {"iter": it, "eta_max": eta_max, "grid_flat": int(flat), "n_atoms": int(w.size)}
        if eta_max > 1.0 + tau:
            thetas = np.vstack([thetas, theta_new[None, :]])
            w = lasso_weights(n, R, psf, y, thetas, lam, fft=fft)
            if not boosted:
                thetas, w = _slide(n, R, psf, y, thetas, w, lam, fft)
            thetas, w = _prune(thetas, w)
            rec["n_atoms"] = int(w.size)
            history.append(rec)
            if log:
                log(rec)
            continue
        if boosted and w.size:
            thetas, w = _slide(n, R, psf, y, thetas, w, lam, fft)
            thetas, w = _prune(thetas, w)
        rec["n_atoms"] = int(w.size)
        history.append(rec)
        if log:
            log(rec)
        break
    th = np.reshape(thetas, (-1, 5))
    C = criterion(n, R, psf, y, th[:, :3], th[:, 3], th[:, 4], w, lam, fft=fft)
    return {"thetas": th, "w": w, "C": C, "history": history}


def sfw(n, R, psf, y, lam, kernels, fft=True, tau=TAU, max_iter=None, log=None):
    """Sliding Frank-Wolfe (Algorithm 1): certificate max, augment, LASSO, slide, prune."""
    return _run(n, R, psf, y, lam, kernels, False, fft, tau, max_iter or 50, log)


def bsfw(n, R, psf, y, lam, kernels, fft=True, tau=TAU, max_iter=None, log=None):
    """Boosted SFW (Algorithm 2): the slide runs once, after the certificate drops below 1."""
    return _run(n, R, psf, y, lam, kernels, True, fft, tau, max_iter or 50, log)
