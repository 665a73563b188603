"""The tensor-core (tcgen05) path: one bf16 MMA tile against numpy, and the certificate of bf16
plans (axis-0 stage on the tensor cores) against the FP64 oracle and the FP32 route.

Tolerances: the tile is exact bf16 products summed in FP32, so it matches the FP64 product of
the same bf16 values to 1e-5 of its largest magnitude.  Certificates on bf16 operands carry
~3 significant digits: 1e-2 of the largest certificate magnitude against the oracle (the
precision configuration's bar); the top-64 voxels re-scored in FP32 seed the oracle's grid
maximum."""

import ctypes

import numpy as np
import pytest

import sfw_inputs
from parity_util import assert_argmax

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_05473_gb300 as m
    m.build_library()
    return m


def _bf16_bits(a):
    """Round float64 values to bfloat16 (nearest even); return the bit patterns and the values."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    back = (r.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return r, back


@pytest.mark.parametrize("K,N,swz", [(16, 16, 0), (64, 32, 0), (192, 32, 0), (96, 48, 0), (256, 128, 0),
                                     (64, 16, 1), (192, 32, 1), (384, 64, 1)])
def test_tensor_core_tile_matches_numpy(sfw, K, N, swz):
    """One MMA tile per operand layout: interleaved 8x8 core matrices, and the 128-byte swizzle
    the certificate pass uses."""
    from paper_2009_05473_gb300 import _abi
    L = _abi.lib()
    L.sfw_test_tc_gemm.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 2 + [ctypes.c_void_p, ctypes.c_int]
    L.sfw_test_tc_gemm.restype = ctypes.c_int
    rng = np.random.default_rng(K * 1000 + N)
    a_bits, a = _bf16_bits(rng.standard_normal((128, K)))
    b_bits, b = _bf16_bits(rng.standard_normal((N, K)))
    a_bits = np.ascontiguousarray(a_bits)
    b_bits = np.ascontiguousarray(b_bits)
    d = np.zeros((128, N), np.float32)
    st = L.sfw_test_tc_gemm(a_bits.ctypes.data, b_bits.ctypes.data, K, N, d.ctypes.data, swz)
    assert st == 0, L.sfw_last_error().decode()
    ref = a @ b.T
    assert np.max(np.abs(d - ref)) <= 1e-5 * np.max(np.abs(ref))


# ragged output rows (n0 not a multiple of 64), kernel counts padded to 16, 32 and 48; all of
# them take the per-axis certificate tail, whose axis-2 inverse also runs on the tensor cores
TC_CASES = [
    ((20, 24, 28), (2, 3, 4), (1.0, 2.0, 3.0), (1.5, 2.0, 2.5)),               # K = 9  -> 16
    ((70, 18, 22), (3, 2, 3), tuple(np.linspace(1, 3, 8)), (1.5, 2.0, 2.5, 3.0)),  # K = 32
    ((33, 40, 16), (2, 4, 2), tuple(np.linspace(1, 3, 10)), (1.5, 2.0, 2.5, 3.0)),  # K = 40 -> 48
    # odd line count x odd half-spectrum length: every other kernel's spectra start off the
    # 16-byte grid, and the last 128-line tile has empty quarters
    ((21, 15, 18), (2, 2, 3), (1.0, 2.0, 3.0), (1.5, 2.5)),                     # K = 6 -> 16
    # one line per 128-column tile (kernels padded to 128)
    ((18, 20, 24), (2, 2, 3), tuple(np.linspace(1, 3, 10)), tuple(np.linspace(1.3, 2.9, 10))),  # K = 100 -> 128
]


@pytest.mark.parametrize("case", TC_CASES)
def test_tensor_core_certificate_matches_oracle(sfw, oracle_mod, case):
    import torch
    n, R, sig, ds = case
    vol = sfw_inputs.make_volume("tc", n, R, (1.2, 1.3, 1.7), 3, seed=21, grid_sigmas=sig, grid_ds=ds,
                                 min_sep=2.0)
    y = np.asarray(oracle_mod.observe(vol, fft=True), np.float32)
    kernels = vol.grid_kernels()
    lam = oracle_mod.lambda_rule(vol.n, vol.R, vol.psf, y.astype(np.float64), kernels, fft=True)
    r = y - np.asarray(oracle_mod.forward(vol.n, vol.R, vol.psf, vol.m[:1], vol.sigma[:1], vol.d[:1],
                                          vol.w[:1], fft=True), np.float32)
    pb = sfw.Plan(vol.n, vol.R, vol.psf, vol.grid_sigmas, vol.grid_ds, precision="bf16")
    pf = sfw.Plan(vol.n, vol.R, vol.psf, vol.grid_sigmas, vol.grid_ds, precision="fp32")
    assert pb.info["tensor_cores"] and not pf.info["tensor_cores"]
    rd = torch.tensor(r, device="cuda")
    sfw._abi.sfw_profile_start(256, None)
    ob = pb.certificate(rd, lam, want_eta=True)
    tags = sfw._abi.sfw_profile_stop()
    # both inverse stages of the certificate ran on the tensor cores
    assert "cert_axis0_tc" in tags and "cert_c2r_tc" in tags, sorted(tags)
    eb = ob["eta"].cpu().numpy()
    ef = pf.certificate(rd, lam, want_eta=True)["eta"].cpu().numpy()
    ref = oracle_mod.eta_grid_fft(vol.n, vol.R, vol.psf, r.astype(np.float64), lam, kernels)
    scale = np.max(np.abs(ref))
    err_b = np.max(np.abs(eb - ref)) / scale
    err_f = np.max(np.abs(ef - ref)) / scale
    print(f"\n[tensor cores {n} K={len(kernels)}] eta rel err: bf16/tcgen05 {err_b:.2e}, fp32 FFT {err_f:.2e}")
    assert err_b <= 1e-2 and err_f <= 1e-5
    # per-voxel max / argk and the grid argmax of the bf16 grid itself are consistent
    assert int(ob["best_idx"].item()) == int(np.argmax(eb))
    np.testing.assert_array_equal(ob["max"].cpu().numpy(), eb.max(axis=0))
    # the FP32 re-score of the top-64 bf16 voxels seeds the oracle's grid maximum
    top = pb.certificate_topk(rd, lam, 64)
    th = top["best_theta"].cpu().numpy()
    vox = int(np.ravel_multi_index(tuple(int(round(x)) for x in th[:3]), vol.n))
    k = int(np.argmin([abs(s - th[3]) + abs(d - th[4]) for s, d in kernels]))
    assert_argmax(k * vol.V + vox, ref, 1e-5 * scale)
    pb.check()
    pb.close()
    pf.close()


def test_tensor_core_engine_choice_by_timing(sfw, oracle_mod, tmp_path):
    """sfw_autotune times the certificate's axis-0 stage on the tensor cores against the FFT
    arithmetic for a bf16 plan, keeps the faster, caches the choice; the certificate stays within
    the bf16 bar of the oracle either way."""
    import torch
    n, R, sig, ds = TC_CASES[1]
    vol = sfw_inputs.make_volume("tc", n, R, (1.2, 1.3, 1.7), 3, seed=21, grid_sigmas=sig, grid_ds=ds,
                                 min_sep=2.0)
    y = np.asarray(oracle_mod.observe(vol, fft=True), np.float32)
    kernels = vol.grid_kernels()
    pb = sfw.Plan(vol.n, vol.R, vol.psf, vol.grid_sigmas, vol.grid_ds, precision="bf16")
    assert pb.info["tensor_cores"]
    cache = str(tmp_path / "engines.txt")
    got = pb.autotune(cache)
    assert got["cert"] == "fft" and got["tensor_cores"] in (True, False)
    again = sfw.Plan(vol.n, vol.R, vol.psf, vol.grid_sigmas, vol.grid_ds, precision="bf16")
    assert again.autotune(cache) == got
    assert open(cache).read().count("|") == 1
    lam = 1.0
    eta = pb.certificate(torch.tensor(y, device="cuda"), lam, want_eta=True)["eta"].cpu().numpy()
    ref = oracle_mod.eta_grid_fft(vol.n, vol.R, vol.psf, y.astype(np.float64), lam, kernels)
    assert np.max(np.abs(eta - ref)) <= 1e-2 * np.max(np.abs(ref))
    pb.close()
    again.close()


def test_more_kernels_than_tensor_core_tiles_fall_back_to_fft(sfw, oracle_mod):
    """K = 130 exceeds the 128 kernels of a tensor-core tile: the bf16 plan keeps the FFT
    arithmetic for the certificate, within the bf16 bar of the oracle."""
    import torch
    vol = sfw_inputs.make_volume("tc", (16, 18, 20), (2, 2, 3), (1.2, 1.3, 1.7), 2, seed=22,
                                 grid_sigmas=tuple(np.linspace(1, 3, 13)), grid_ds=tuple(np.linspace(1.3, 2.9, 10)),
                                 min_sep=2.0)
    y = np.asarray(oracle_mod.observe(vol, fft=True), np.float32)
    kernels = vol.grid_kernels()
    assert len(kernels) == 130
    pb = sfw.Plan(vol.n, vol.R, vol.psf, vol.grid_sigmas, vol.grid_ds, precision="bf16")
    assert not pb.info["tensor_cores"]
    eta = pb.certificate(torch.tensor(y, device="cuda"), 1.0, want_eta=True)["eta"].cpu().numpy()
    ref = oracle_mod.eta_grid_fft(vol.n, vol.R, vol.psf, y.astype(np.float64), 1.0, kernels)
    assert np.max(np.abs(eta - ref)) <= 1e-2 * np.max(np.abs(ref))
    pb.close()
