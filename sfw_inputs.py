"""Seeded synthetic inputs for the sliding Frank-Wolfe hot path.

This module is shared by the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2009_05473_gb300``).  It only draws random numbers and builds the
given data of the inverse problem (the PSF H, the atom set of the ground-truth
measure mu*, a unit-variance noise field and the certificate grid).  It holds
none of the method's arithmetic: rendering, convolution, the criterion, the
certificate and every solver step live on each side separately.

Workloads stand in for the paper's synthetic volumes (Section 3: 60^3 to 100^3
voxels, 4 to 8 atoms, white Gaussian noise, a PSF that blurs about twice as
much along the optical axis).  The paper's tomographic-microscopy PSF is not
available, so an anisotropic Gaussian with the axial width twice the lateral
one stands in for it (rotation-invariant about axis 2, as the paper's Fig. 1
caption states for its PSF).

Conventions (the paper is silent on them):
  * a volume of shape (n0, n1, n2) is C-contiguous, axis 2 fastest;
  * voxel centres sit at integer coordinates 0..n_a-1;
  * the PSF has shape (2R0+1, 2R1+1, 2R2+1), is centred at index R and sums
    to one;
  * atom parameters are drawn per atom in the order m (3 uniform in the inner
    box that leaves a 4-voxel margin), sigma, d, w; m is redrawn until it lies
    at least ``min_sep`` voxels from every earlier atom; the noise field is
    drawn last, in C order, from the same generator.
"""

from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np

MARGIN = 4


@dataclasses.dataclass
class Volume:
    """One synthetic deconvolution problem (inputs only, no derived data)."""

    name: str
    n: Tuple[int, int, int]
    R: Tuple[int, int, int]
    psf_sigma: Tuple[float, float, float]
    psf: np.ndarray            # float64, (2R+1) box, sums to 1
    m: np.ndarray              # float64 (N, 3), grid coordinates
    sigma: np.ndarray          # float64 (N,)
    d: np.ndarray              # float64 (N,)
    w: np.ndarray              # float64 (N,)
    noise: np.ndarray          # float64 standard normal, shape n
    noise_frac: float          # noise std = noise_frac * max(noise-free y)
    grid_sigmas: np.ndarray    # certificate grid, sigma values
    grid_ds: np.ndarray        # certificate grid, d values
    lambda_frac: float = 0.05  # lambda = lambda_frac * max over the grid of Phi^T y
    seed: int = 0

    @property
    def N(self) -> int:
        return int(self.w.shape[0])

    @property
    def V(self) -> int:
        return int(np.prod(self.n))

    @property
    def K(self) -> int:
        return int(len(self.grid_sigmas) * len(self.grid_ds))

    def grid_kernels(self) -> List[Tuple[float, float]]:
        """Certificate-grid kernels (sigma_k, d_k), k = i_sigma * n_d + i_d."""
        return [(float(s), float(dd)) for s in self.grid_sigmas for dd in self.grid_ds]


def gaussian_psf(psf_sigma, R) -> np.ndarray:
    """Sampled anisotropic Gaussian on a (2R+1) box, centred, normalised to sum 1."""
    axes = [np.exp(-0.5 * (np.arange(-r, r + 1, dtype=np.float64) / s) ** 2)
            for s, r in zip(psf_sigma, R)]
    h = axes[0][:, None, None] * axes[1][None, :, None] * axes[2][None, None, :]
    return h / h.sum()


def tilted_gaussian_psf(psf_sigma, R, angles) -> np.ndarray:
    """Sampled anisotropic Gaussian whose principal axes are turned by angles[0] about axis 0
    and then angles[1] about axis 1 (radians): covariance Q diag(sigma^2) Q^T on a (2R+1) box,
    centred, normalised to sum 1.  Not separable along the grid axes; point-symmetric."""
    a, b = angles
    r0 = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
    r1 = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
    q = r1 @ r0
    prec = q @ np.diag(1.0 / np.asarray(psf_sigma, np.float64) ** 2) @ q.T
    x = np.stack(np.meshgrid(*[np.arange(-r, r + 1, dtype=np.float64) for r in R], indexing="ij"), -1)
    h = np.exp(-0.5 * np.einsum("...i,ij,...j->...", x, prec, x))
    return h / h.sum()


def _draw_atoms(rng, n, N, sigma_rng, d_rng, w_rng, min_sep):
    lo = np.full(3, float(MARGIN))
    hi = np.array(n, dtype=np.float64) - 1.0 - MARGIN
    m = np.zeros((N, 3))
    sig = np.zeros(N)
    dd = np.zeros(N)
    w = np.zeros(N)
    for i in range(N):
        for _ in range(100000):
            cand = rng.uniform(lo, hi)
            if i == 0 or min_sep <= 0 or np.min(np.linalg.norm(m[:i] - cand, axis=1)) >= min_sep:
                break
        else:  # pragma: no cover - the configured boxes are far from full
            raise RuntimeError("could not place atoms with the requested separation")
        m[i] = cand
        sig[i] = rng.uniform(*sigma_rng)
        dd[i] = rng.uniform(*d_rng)
        w[i] = rng.uniform(*w_rng)
    return m, sig, dd, w


def make_volume(name: str, n, R, psf_sigma, N, *, seed=0, noise_frac=0.02, psf=None,
                grid_sigmas=(1.0, 2.0, 3.0), grid_ds=(2.0,), sigma_rng=(1.0, 3.0),
                d_rng=(1.5, 2.5), w_rng=(0.5, 1.5), min_sep=4.0, rng=None) -> Volume:
    rng = np.random.default_rng(seed) if rng is None else rng
    n = tuple(int(v) for v in n)
    R = tuple(int(v) for v in R)
    m, sig, dd, w = _draw_atoms(rng, n, N, sigma_rng, d_rng, w_rng, min_sep)
    noise = rng.standard_normal(n)
    return Volume(name=name, n=n, R=R, psf_sigma=tuple(float(s) for s in psf_sigma),
                  psf=gaussian_psf(psf_sigma, R) if psf is None else np.asarray(psf, np.float64),
                  m=m, sigma=sig, d=dd, w=w, noise=noise,
                  noise_frac=float(noise_frac), grid_sigmas=np.asarray(grid_sigmas, np.float64),
                  grid_ds=np.asarray(grid_ds, np.float64), seed=seed)


# --- the workloads, named by what they are -------------------------------------------

ANISO_PSF = (1.5, 1.5, 3.0)
ANISO_R = (7, 7, 15)  # 15 x 15 x 31 support


def vol32_iso_n3(seed=0) -> Volume:
    """32^3, isotropic PSF sigma 1.5 on 9^3, N=3, grid sigma in {1,2,3} x d=2 (K=3)."""
    return make_volume("vol32_iso9_n3_k3", (32, 32, 32), (4, 4, 4), (1.5, 1.5, 1.5), 3,
                       seed=seed, noise_frac=0.01, grid_sigmas=(1.0, 2.0, 3.0), grid_ds=(2.0,))


def vol64_aniso_n10(seed=0) -> Volume:
    """64^3, PSF sigma (1.5,1.5,3) on 15x15x31, N=10, 5 sigma x 3 d grid (K=15)."""
    return make_volume("vol64_aniso_n10_k15", (64, 64, 64), ANISO_R, ANISO_PSF, 10, seed=seed,
                       noise_frac=0.02, grid_sigmas=np.linspace(1.0, 3.0, 5),
                       grid_ds=(1.5, 2.0, 2.5))


def vol128_aniso_n30(seed=0) -> Volume:
    """128^3, same PSF, N=30, 8 sigma x 4 d grid (K=32)."""
    return make_volume("vol128_aniso_n30_k32", (128, 128, 128), ANISO_R, ANISO_PSF, 30,
                       seed=seed, noise_frac=0.02, grid_sigmas=np.linspace(1.0, 3.0, 8),
                       grid_ds=np.linspace(1.5, 2.5, 4))


def vol256x256x64_n100(seed=0) -> Volume:
    """256x256x64, same PSF, N=100 atoms with w in U[0.2, 2] (sliding-step workload)."""
    return make_volume("vol256x256x64_n100", (256, 256, 64), ANISO_R, ANISO_PSF, 100,
                       seed=seed, noise_frac=0.02, grid_sigmas=np.linspace(1.0, 3.0, 5),
                       grid_ds=(1.5, 2.0, 2.5), w_rng=(0.2, 2.0))


BATCH_SHAPES = ((48, 48, 48), (64, 64, 64), (96, 96, 64), (128, 128, 128))


def batch_volume(i: int) -> Volume:
    """Volume i of the uneven batch: seed 1000+i draws shape, N, PSF widths, atoms, noise."""
    rng = np.random.default_rng(1000 + i)
    shape = BATCH_SHAPES[int(rng.integers(len(BATCH_SHAPES)))]
    N = int(rng.integers(5, 41))
    lat = float(rng.uniform(1.2, 2.0))
    ax = float(rng.uniform(2.5, 3.5))
    return make_volume(f"batch{i}", shape, ANISO_R, (lat, lat, ax), N, seed=1000 + i,
                       noise_frac=0.02, grid_sigmas=np.linspace(1.0, 3.0, 5),
                       grid_ds=(1.5, 2.0, 2.5), rng=rng)


def batch_uneven(count: int = 64) -> List[Volume]:
    """The uneven batch: ``count`` volumes from {48^3, 64^3, 96x96x64, 128^3}, N in U{5..40}."""
    return [batch_volume(i) for i in range(count)]


def random_atoms(rng, n, N, sigma_rng=(1.0, 3.0), d_rng=(1.5, 2.5), w_rng=(0.5, 1.5),
                 margin=MARGIN):
    """Unconstrained atom draw for parity tests (m may come close to each other)."""
    lo = np.full(3, float(margin))
    hi = np.array(n, dtype=np.float64) - 1.0 - margin
    m = rng.uniform(lo, hi, size=(N, 3))
    return m, rng.uniform(*sigma_rng, N), rng.uniform(*d_rng, N), rng.uniform(*w_rng, N)


def vol64_tilted_n10(seed=0) -> Volume:
    """The 64^3 workload with a non-separable PSF: the (1.5, 1.5, 3) Gaussian turned by 0.5 rad
    about axis 0 and 0.3 rad about axis 1, on the same 15x15x31 support."""
    return make_volume("vol64_tilted_n10_k15", (64, 64, 64), ANISO_R, ANISO_PSF, 10, seed=seed,
                       noise_frac=0.02, psf=tilted_gaussian_psf(ANISO_PSF, ANISO_R, (0.5, 0.3)),
                       grid_sigmas=np.linspace(1.0, 3.0, 5), grid_ds=(1.5, 2.0, 2.5))


WORKLOADS = {
    "vol32_iso9_n3_k3": vol32_iso_n3,
    "vol64_aniso_n10_k15": vol64_aniso_n10,
    "vol64_tilted_n10_k15": vol64_tilted_n10,
    "vol128_aniso_n30_k32": vol128_aniso_n30,
    "vol256x256x64_n100": vol256x256x64_n100,
}
