"""sfw_argmax_noalloc: the arg-maximum / top-k for callers that cannot allocate device memory.

Callers whose device memory belongs to another allocator or a fixed budget, and loops that must
not let the cudaFree of a re-allocation synchronise the device, cannot use a routine that
allocates its own scratch.  sfw_argmax_noalloc uses a static device array of the library
instead.  This test calls it through the C ABI twice in a row (different sizes and top-k, so
stale scratch contents from the first call would show up in the second) and checks each result
against sfw_argmax, the entry point that allocates.  Results are index work: they must match
exactly.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_05473_gb300 as sfw
    sfw.build_library()
    return torch, sfw._abi


def _run(torch, abi, fn, v, topk):
    vals = torch.empty(topk, dtype=torch.float32, device="cuda")
    idx = torch.empty(topk, dtype=torch.int64, device="cuda")
    fn(v.data_ptr(), v.numel(), topk, vals.data_ptr(), idx.data_ptr(),
       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return vals.cpu().numpy(), idx.cpu().numpy()


def _data(seed, count, ties=5):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(count).astype(np.float32)
    picks = rng.choice(count, ties, replace=False)
    v[picks] = v.max() + 1.0
    return v


def test_noalloc_matches_allocating_argmax_two_calls(env):
    torch, abi = env
    cases = [(_data(1, 3_000_017), 64), (_data(2, 70_001), 1), (_data(3, 4_099), 8)]
    for v_np, k in cases:
        v = torch.tensor(v_np, device="cuda")
        ref_vals, ref_idx = _run(torch, abi, abi.sfw_argmax, v, k)
        got_vals, got_idx = _run(torch, abi, abi.sfw_argmax_noalloc, v, k)
        np.testing.assert_array_equal(got_idx, ref_idx)
        np.testing.assert_array_equal(got_vals, ref_vals)
        order = np.lexsort((np.arange(v_np.size), -v_np.astype(np.float64)))[:k]
        np.testing.assert_array_equal(got_idx, order)


def test_noalloc_reports_nan_and_rejects_oversize(env):
    torch, abi = env
    v = torch.zeros(10_000, device="cuda")
    v[1234] = float("nan")
    _, idx = _run(torch, abi, abi.sfw_argmax_noalloc, v, 4)
    assert idx[0] == -1
    # 64 keys per 4096-value block over 2^23 + 1 values exceeds the static scratch
    big = torch.zeros((1 << 23) + 1, device="cuda")
    with pytest.raises(abi.SfwError) as e:
        _run(torch, abi, abi.sfw_argmax_noalloc, big, 64)
    assert e.value.status == 2
    _, idx = _run(torch, abi, abi.sfw_argmax_noalloc, big, 1)   # top-1 has no size limit
    assert idx[0] == 0
