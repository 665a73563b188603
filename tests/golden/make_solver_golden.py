"""Writes tests/golden/vol64_solvers.json: the FP64 oracle's SFW (Algorithm 1) and BSFW
(Algorithm 2) on the 64^3 workload (seed 0; PSF sigma (1.5, 1.5, 3) on 15 x 15 x 31; 10 atoms;
grid 5 sigma x 3 d), a frozen record for the GPU solver's parity test.  The observation is the
oracle's (Fourier-domain blur, 2 % noise) rounded to FP32, the bytes the GPU path also gets;
lambda = 0.05 max_grid Phi^T y (the lambda rule).  Calls only ``oracle`` and the seeded
generators of ``sfw_inputs``; takes tens of minutes on CPU.

    python tests/golden/make_solver_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import sfw_inputs  # noqa: E402


def observation():
    vol = sfw_inputs.vol64_aniso_n10(seed=0)
    y = oracle.observe(vol, fft=True).astype(np.float32).astype(np.float64)
    return vol, y


def solve(vol, y, lam, boosted):
    n, R, kernels = vol.n, vol.R, vol.grid_kernels()
    t0 = time.time()
    out = (oracle.bsfw if boosted else oracle.sfw)(
        n, R, vol.psf, y, lam, kernels, fft=True,
        log=lambda rec: print(("bsfw" if boosted else "sfw"), rec, f"{time.time() - t0:.0f}s", flush=True))
    return {"atoms": int(out["w"].size), "C": float(out["C"]),
            "seeds": [int(h["grid_flat"]) for h in out["history"]],
            "eta_max": [float(h["eta_max"]) for h in out["history"]],
            "thetas": out["thetas"].tolist(), "w": out["w"].tolist(), "seconds": time.time() - t0}


def main():
    oracle.build_oracle()
    vol, y = observation()
    kernels = vol.grid_kernels()
    lam = oracle.lambda_rule(vol.n, vol.R, vol.psf, y, kernels, fft=True)
    rec = {
        "case": {"workload": "vol64_aniso_n10 seed 0", "n": list(vol.n), "R": list(vol.R),
                 "kernels": kernels, "lambda": lam, "tau": oracle.TAU,
                 "recipe": "y = oracle.observe(vol64_aniso_n10(seed=0), fft=True) rounded to FP32; "
                           "lambda = oracle.lambda_rule(..., fft=True) (0.05 x grid max of Phi^T y)"},
        "citations": {"sfw": "Algorithm 1 (certificate maximum, augment, LASSO, slide, prune)",
                      "bsfw": "Algorithm 2 (slide only once the certificate drops below 1)",
                      "seeds": "flat grid index k V + lin(m) of the grid maximum at every outer iteration "
                               "(step 1), ties to the lowest",
                      "eta_max": "certificate maximum after the local ascent (Eq. 5)",
                      "C": "Eq. 4 at the returned measure"},
        "sfw": solve(vol, y, lam, False),
        "bsfw": solve(vol, y, lam, True),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vol64_solvers.json")
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(path)


if __name__ == "__main__":
    main()
