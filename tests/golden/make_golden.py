"""Writes tests/golden/tiny_13x11x9.json: the FP64 oracle's values on one small seeded case
(13 x 11 x 9 grid, half-widths (2, 3, 1), three atoms, an asymmetric PSF), as a frozen record
of the oracle.  Calls only ``oracle`` and the seeded generators of ``sfw_inputs``.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import sfw_inputs  # noqa: E402

N = (13, 11, 9)
R = (2, 3, 1)
KERNELS = [(1.0, 1.5), (1.0, 2.0), (2.0, 2.5)]
LAM = 0.2   # the fixed regularisation weight of the paper's experiments (Section 4)


def case():
    vol = sfw_inputs.make_volume("golden", N, R, (1.1, 1.4, 0.9), 3, seed=7, grid_sigmas=(1.0, 2.0),
                                 grid_ds=(1.5, 2.0, 2.5), min_sep=2.0)
    rng = np.random.default_rng(17)
    psf = vol.psf * (1.0 + 0.3 * rng.random(vol.psf.shape))
    psf /= psf.sum()
    y = oracle.forward(N, R, psf, vol.m, vol.sigma, vol.d, vol.w)
    y = y + 0.01 * np.max(y) * rng.standard_normal(y.shape)
    # a perturbed estimate, so that the residual, the gradient and eta are all non-trivial
    m = vol.m + np.array([[0.3, -0.2, 0.1]])
    return psf, y, m, vol.sigma * 1.1, np.clip(vol.d + 0.1, 1.3, 2.9), vol.w * 0.8


def values():
    psf, y, m, s, d, w = case()
    C, g, r = oracle.loss_and_grad(N, R, psf, y, m, s, d, w, LAM, fft=False)
    eta = oracle.eta_grid(N, R, psf, r, LAM, KERNELS)
    k, best = oracle.grid_argmax(eta)
    return {
        "forward_sum": float(np.sum(oracle.forward(N, R, psf, m, s, d, w))),
        "forward_sample": [float(v) for v in oracle.forward(N, R, psf, m, s, d, w).ravel()[::97]],
        "criterion": float(C),
        "gradient": [float(v) for v in np.asarray(g).ravel()],
        "eta_max": float(best),
        "eta_argmax": int(k),
        "eta_sample": [float(v) for v in np.asarray(eta).ravel()[::131]],
    }


def main():
    rec = {
        "case": {"n": N, "R": R, "kernels": KERNELS, "lambda": LAM,
                 "recipe": "sfw_inputs.make_volume('golden', n, R, (1.1, 1.4, 0.9), 3, seed=7) with the PSF "
                           "scaled by 1 + 0.3 U(0,1) (seed 17, renormalised), 1 % Gaussian noise, "
                           "estimate = truth shifted by (0.3, -0.2, 0.1), sigma x 1.1, d + 0.1, w x 0.8"},
        "citations": {"forward_sum": "Eq. 3 (observation model, Eq. 2 atoms)",
                      "forward_sample": "Eq. 3, every 97th voxel",
                      "criterion": "Eq. 4",
                      "gradient": "Eq. 4, analytic gradient (Section 2): dC/dm (3 per atom), then dC/dsigma, dC/dd, dC/dw (one per atom each)",
                      "eta_max": "Eq. 5 on the grid of Algorithm 1 step 1",
                      "eta_argmax": "flat index k * V + voxel, ties to the lowest",
                      "eta_sample": "Eq. 5, every 131st (kernel, voxel)"},
        "values": values(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_13x11x9.json")
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(path)


if __name__ == "__main__":
    main()
