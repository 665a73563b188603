"""The SFW / BSFW host loop of the GPU solver (``solver.GPUSolver``: certificate maximum and
local ascent, LASSO on the Gram form, sliding descent, pruning, stopping test) driven by an
FP64 test double of the plan built from the oracle's operators, against the oracle's own
Algorithms 1 and 2 on a small seeded volume: same atoms, same criterion.  CPU only."""

import numpy as np
import pytest
import torch

import sfw_inputs


class _Atoms:
    def __init__(self, m, sigma, d, w):
        self.m = np.reshape(np.asarray(m, np.float64), (-1, 3))
        self.sigma = np.asarray(sigma, np.float64).ravel()
        self.d = np.asarray(d, np.float64).ravel()
        self.w = np.asarray(w, np.float64).ravel()
        self.N = self.w.size

    @staticmethod
    def from_numpy(m, sigma, d, w, device=None):
        return _Atoms(m, sigma, d, w)


class _OraclePlan:
    """The plan's methods that the solver calls, computed by the FP64 oracle on the host."""

    def __init__(self, oracle, vol):
        self.o, self.n, self.R, self.psf = oracle, tuple(vol.n), tuple(vol.R), vol.psf
        self.kernels = [tuple(k) for k in vol.grid_kernels()]
        self.V = int(np.prod(self.n))
        self.K = len(self.kernels)

    def _np(self, t):
        return t.detach().cpu().numpy().astype(np.float64) if torch.is_tensor(t) else np.asarray(t, np.float64)

    def slide_loss_grad(self, y, a, lam, want_residual=False, want_grad=True):
        C, g, r = self.o.loss_and_grad(self.n, self.R, self.psf, self._np(y), a.m, a.sigma, a.d, a.w, lam, fft=True)
        return (torch.tensor([C], dtype=torch.float64), torch.tensor(g),
                torch.tensor(r) if want_residual else None)

    def certificate(self, r, lam, want_max=False):
        eta = self.o.eta_grid_fft(self.n, self.R, self.psf, self._np(r), lam, self.kernels)
        flat, val = self.o.grid_argmax(eta)
        return {"best_idx": torch.tensor([flat]), "best_val": torch.tensor([val])}

    def eta_points(self, r, lam, theta):
        b = self.o.backproject_fft(self.n, self.R, self.psf, self._np(r))
        e, g = self.o.eta_points(self.n, self.R, b, lam, np.asarray(theta, np.float64), with_grad=True)
        return torch.tensor(e), torch.tensor(g)

    def gram(self, a, y):
        th = np.concatenate([a.m, a.sigma[:, None], a.d[:, None]], 1)
        A = self.o.atom_columns(self.n, self.R, self.psf, th, fft=True)
        return torch.tensor(A @ A.T), torch.tensor(A @ self._np(y).ravel())


@pytest.fixture()
def host_solver(monkeypatch):
    from paper_2009_05473_gb300 import solver
    monkeypatch.setattr(solver, "AtomSet", _Atoms)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    return solver


def _case(oracle_mod):
    vol = sfw_inputs.make_volume("loop", (16, 16, 14), (2, 2, 3), (1.2, 1.2, 1.8), 2, seed=3,
                                 grid_sigmas=(1.0, 2.0), grid_ds=(2.0,), min_sep=5.0, noise_frac=0.005)
    y = oracle_mod.observe(vol, fft=True)
    lam = oracle_mod.lambda_rule(vol.n, vol.R, vol.psf, y, vol.grid_kernels(), frac=0.15, fft=True)
    return vol, y, lam


@pytest.mark.parametrize("boosted", [False, True])
def test_host_loop_matches_oracle_algorithm(oracle_mod, host_solver, boosted):
    vol, y, lam = _case(oracle_mod)
    plan = _OraclePlan(oracle_mod, vol)
    ref = (oracle_mod.bsfw if boosted else oracle_mod.sfw)(vol.n, vol.R, vol.psf, y, lam, vol.grid_kernels())
    out = host_solver.GPUSolver(plan, torch.tensor(y), lam).run(boosted=boosted)
    # the same greedy path: the grid maximum that seeds every outer iteration.  Once the
    # certificate's excess over 1 is within a few 1e-3, the two ascents' tolerances may pick
    # different near-duplicate points (BSFW keeps adding such atoms until its final slide),
    # so the paths are compared while the excess is clear
    V = plan.V
    seeds = []
    for h in out["history"]:
        th = np.asarray(h["seed"])
        k = plan.kernels.index((float(th[3]), float(th[4])))
        seeds.append(k * V + int(np.ravel_multi_index(tuple(int(round(v)) for v in th[:3]), plan.n)))
    clear = [i for i, h in enumerate(ref["history"]) if h["eta_max"] > 1.01]
    assert clear and [seeds[i] for i in clear] == [ref["history"][i]["grid_flat"] for i in clear]
    if not boosted:
        # SFW slides after every addition: the same path, atoms and criterion
        assert seeds == [h["grid_flat"] for h in ref["history"]]
        assert out["w"].size == ref["w"].size
        order = np.argsort(ref["thetas"][:, 0])
        got = np.argsort(out["thetas"][:, 0])
        assert np.allclose(out["thetas"][got, :3], ref["thetas"][order, :3], atol=2e-2)
        assert np.allclose(out["w"][got], ref["w"][order], rtol=2e-2)
        assert abs(out["C"] - ref["C"]) <= 1e-6 * abs(ref["C"])
    else:
        assert abs(out["C"] - ref["C"]) <= 1e-3 * abs(ref["C"])
    # every outer iteration but the last added an atom whose certificate exceeded 1 + tau
    assert all(h["eta_max"] > 1.0 for h in out["history"][:-1])
    assert out["history"][-1]["eta_max"] <= 1.0 + 1e-3


def test_lambda_path_host_logic(oracle_mod, host_solver):
    """lambda_max is step 1 of Algorithm 1 on y at lambda = 1 (the oracle's own step 1 gives
    the same value); above it the measure stays empty; along decreasing lambda each warm-started
    solve ends with the certificate at most 1 + tau and a criterion of its own lambda."""
    vol, y, _ = _case(oracle_mod)
    plan = _OraclePlan(oracle_mod, vol)
    yt = torch.tensor(y)
    lmax = host_solver.lambda_max(plan, yt)
    _, eta_ref, _ = oracle_mod.oracle._certificate_max(vol.n, vol.R, vol.psf, y, np.zeros((0, 5)), np.zeros(0), 1.0,
                                                plan.kernels, True)
    assert abs(lmax - eta_ref) <= 1e-6 * eta_ref
    path = host_solver.lambda_path(plan, yt, fractions=(1.01, 0.3, 0.15), boosted=False)
    assert [p["fraction"] for p in path] == [1.01, 0.3, 0.15]
    assert path[0]["w"].size == 0
    assert path[1]["w"].size >= 1 and path[2]["w"].size >= path[1]["w"].size
    for p in path:
        assert p["history"][-1]["eta_max"] <= 1.0 + 1e-3
        th = p["thetas"]
        C = oracle_mod.criterion(vol.n, vol.R, vol.psf, y, th[:, :3], th[:, 3], th[:, 4], p["w"], p["lambda"],
                                 fft=True)
        assert abs(p["C"] - C) <= 1e-9 * max(1.0, abs(C))
