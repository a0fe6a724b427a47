"""svt_polar_noalloc: the solve with library-owned static scratch, for callers
that cannot allocate device memory. Collected last on purpose, so that a run
stopping at the first failure has already run every other test.

Its output must match the ordinary entry point (svt_polar_ex with a caller
workspace) within the tolerance the batch/serving tests use for "same solve"
(1e-5 relative), on calls in a row with different shapes and then the first shape
again (the shared array keeps the previous call's contents, so the cached plan of
the first shape runs over what the second left there), and all must stay within
the BF16 tier's 2e-2 of the FP64 oracle. Once a shape has been solved, a further
call allocates nothing on the device: the driver's free-memory count and torch's
allocator counters are the same before and after it."""
import numpy as np
import pytest
import torch

import oracle
import svt_workloads as wl

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2607_22484_gb300")


def _gap_matrix(m, n, seed, tau=0.3):
    k = min(m, n)
    rng = np.random.default_rng(seed)
    lo = np.sort(rng.uniform(0.01, tau - 0.06, k // 2))
    hi = np.sort(rng.uniform(tau + 0.06, 1.0, k - k // 2 - 1))
    sig = np.sort(np.concatenate([lo, hi, [1.0]]))[::-1]
    return wl.spectrum_matrix(sig, m, n, seed)


def test_noalloc_matches_svt_polar_two_calls():
    ctx = pkg.Context(0, workspace_bytes=64 << 20)
    for shape, seed in (((256, 192), 1), ((100, 300), 2), ((256, 192), 1)):
        a = _gap_matrix(*shape, seed=seed)
        dev = torch.from_numpy(a).cuda()
        out = torch.full_like(dev, float("nan"))
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        pkg.polar_noalloc(dev, 0.3, out=out, status=status, iters=20, prec="bf16")
        ref = ctx.polar(dev, 0.3, iters=20, prec="bf16")
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = out.cpu().numpy().astype(np.float64)
        assert oracle.relerr(got, ref.cpu().numpy()) < 1e-5
        exact = oracle.svt_definition(a.astype(np.float64), 0.3)
        assert oracle.relerr(got, exact) < 2e-2


def test_noalloc_rejects_sizes_beyond_scratch():
    a = torch.zeros(2048, 2048, device="cuda")
    with pytest.raises(pkg.SVTError) as e:
        pkg.polar_noalloc(a, 0.5, out=torch.empty_like(a))
    assert e.value.status == pkg.binding.ERR_UNSUPPORTED


def test_noalloc_second_call_allocates_nothing():
    import gc
    a = torch.from_numpy(_gap_matrix(300, 260, seed=4)).cuda()
    out = torch.empty_like(a)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    pkg.polar_noalloc(a, 0.3, out=out, status=status, iters=20, prec="bf16")  # plan, modules
    # Earlier tests' tensors must not be collected in the middle of the measurement.
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        free0, _ = torch.cuda.mem_get_info()
        alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
        for _ in range(3):
            pkg.polar_noalloc(a, 0.3, out=out, status=status, iters=20, prec="bf16")
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    finally:
        gc.enable()
    assert int(status.item()) == 0
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0
