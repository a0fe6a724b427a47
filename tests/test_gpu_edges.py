"""Edge cases of the GPU solve through the C ABI: vectors and tiny matrices, the zero
matrix, tau on a singular value, strided input/output, and argument limits."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2607_22484_gb300")


@pytest.fixture(scope="module")
def ctx():
    return pkg.Context(0, workspace_bytes=16 << 20)


def _solve(ctx, a, tau, **opts):
    dev = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    y = ctx.polar(dev, tau, status=st, **opts)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64), int(st.item())


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (2, 3), (3, 3), (65, 1)])
@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp64"])
def test_tiny_and_vector_shapes(ctx, shape, prec):
    rng = np.random.default_rng(sum(shape))
    a = rng.standard_normal(shape)
    s = np.linalg.svd(a, compute_uv=False)
    # tau strictly inside the widest gap of the spectrum (or below sigma_max for rank 1)
    cand = np.concatenate([[0.0], np.sort(s)])
    i = int(np.argmax(np.diff(cand)))
    tau = 0.5 * (cand[i] + cand[i + 1])
    exact, (u, sig, v) = oracle.svt_definition(a.astype(np.float32).astype(np.float64), tau,
                                               return_svd=True)
    y, st = _solve(ctx, a, tau, iters=30, prec=prec, schedule="ns3" if prec == "fp64" else "pe5")
    assert st == 0
    if oracle.gap(sig, tau) >= 0.05:
        # FP64 tier: 1e-9 plus the FP32 output's rounding floor (~6e-8)
        tol = {"bf16": 2e-2, "fp32": 1e-4, "fp64": 1e-9 + 1e-7}[prec]
        assert oracle.relerr(y, exact, a) < tol
        if prec == "fp64":  # the FP64 result itself, at the FP32 tau the ABI carries
            dev = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
            y64 = ctx.polar_f64(dev, tau, iters=30, schedule="ns3")
            torch.cuda.synchronize()
            tau32 = float(np.float32(tau))
            exact32 = oracle.svt_definition(a.astype(np.float32).astype(np.float64), tau32)
            assert oracle.relerr(y64.cpu().numpy(), exact32, a) < 1e-9


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp64"])
def test_zero_matrix(ctx, prec):
    y, st = _solve(ctx, np.zeros((40, 24)), 0.3, iters=10, prec=prec)
    assert st == 0
    assert np.all(y == 0)


def test_tau_on_a_singular_value(ctx):
    """sigma = tau contributes (sigma - tau) = 0 either way: the result stays finite
    and equals the SVT of the other singular values."""
    rng = np.random.default_rng(3)
    q1 = np.linalg.qr(rng.standard_normal((32, 32)))[0]
    q2 = np.linalg.qr(rng.standard_normal((32, 32)))[0]
    sig = np.concatenate([[1.0, 0.8], np.full(1, 0.5), np.linspace(0.2, 0.01, 29)])
    a = (q1 * sig) @ q2.T
    y, st = _solve(ctx, a, 0.5, iters=30, prec="fp32")
    assert st == 0 and np.all(np.isfinite(y))
    exact = (q1 * np.maximum(sig - 0.5, 0)) @ q2.T
    # the sigma = tau term's eigenvalue of the shifted Gram is 0: the odd iteration keeps
    # it at 0, so its weight is 1/2 (sigma - tau) = 0 -- the error stays small
    assert oracle.relerr(y, exact) < 1e-3


def test_strided_input_and_output(ctx):
    rng = np.random.default_rng(8)
    m, n = 150, 110
    base = torch.from_numpy(rng.standard_normal((m, n + 13)).astype(np.float32)).cuda()
    A = base[:, 5:5 + n]  # lda = n + 13, unaligned start
    outbase = torch.full((m, n + 7), 7.0, device="cuda")
    Y = outbase[:, 3:3 + n]
    s = np.linalg.svd(A.cpu().numpy().astype(np.float64), compute_uv=False)
    tau = float(np.median(s))
    ctx.polar(A, tau, out=Y, iters=20, prec="fp32")
    torch.cuda.synchronize()
    exact = oracle.svt_definition(A.cpu().numpy().astype(np.float64), tau)
    assert oracle.relerr(Y.cpu().numpy(), exact) < 1e-3  # no gap guarantee: loose
    # columns outside Y untouched
    ob = outbase.cpu().numpy()
    assert np.all(ob[:, :3] == 7.0) and np.all(ob[:, 3 + n:] == 7.0)


def test_argument_limits(ctx):
    a = torch.zeros(8, 8, device="cuda")
    with pytest.raises(pkg.SVTError) as e:
        ctx.polar(a[:, :0], 0.1)
    assert e.value.status == pkg.binding.ERR_INVALID
    big = torch.zeros(4100, 16, device="cuda")
    with pytest.raises(pkg.SVTError) as e:
        ctx.polar(big, 0.1, prec="fp64")
    assert e.value.status == pkg.binding.ERR_UNSUPPORTED
    with pytest.raises(pkg.SVTError) as e:
        ctx.polar(a, 0.1, ell0=1.5)
    assert e.value.status == pkg.binding.ERR_INVALID


# --- the largest row count the API accepts: 2^20 x 1024 (and its transpose)
#
# 2^30 elements: the BF16 copies of X0 are 2 GiB and the FP32 input and output 4 GiB,
# so every element offset and byte offset above 2^31 is exercised. The input has a
# known SVD built from cheap exact pieces: U stacks 1024 blocks S_b Q / 32 (Q a random
# 1024 x 1024 orthogonal matrix, S_b random sign diagonals), so U^T U = sum_b Q^T Q /
# 1024 = I; A = U diag(sigma) V^T is then the stack of S_b B / 32 with
# B = Q diag(sigma) V^T, and A_tau the stack of S_b B_tau / 32 with
# B_tau = Q diag(max(sigma - tau, 0)) V^T (Eq. 1). Sign flips and the power-of-two
# scale are exact, so B and B_tau (NumPy, FP64) fix every entry.

def _stacked_known(seed):
    rng = np.random.default_rng(seed)
    n = 1024
    sig = np.concatenate([rng.uniform(0.36, 1.0, 100), rng.uniform(0.0, 0.24, n - 100)])
    sig[0] = 1.0
    q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    v = np.linalg.qr(rng.standard_normal((n, n)))[0]
    b = (q * sig) @ v.T
    b_tau = (q * np.maximum(sig - 0.3, 0.0)) @ v.T
    signs = rng.choice(np.array([-1.0, 1.0], dtype=np.float32), size=(n, n))  # S_b diagonals
    return b, b_tau, signs


@pytest.mark.parametrize("wide", [False, True])
def test_largest_row_count(ctx, wide):
    nb, n = 1024, 1024
    b, b_tau, signs = _stacked_known(31 + wide)
    sgn = torch.from_numpy(signs).cuda()                      # (block, row) -> sign
    blk = torch.from_numpy((b / 32.0).astype(np.float32)).cuda()
    # A (tall): rows b * 1024 + i are signs[b, i] * B[i, :] / 32; the wide case is A^T.
    a = (sgn[:, :, None] * blk[None, :, :]).reshape(nb * n, n)
    if wide:
        a = a.T.contiguous()
    ctx.ensure_workspace(pkg.workspace_bytes(a.shape[0], a.shape[1], prec="bf16"))
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    y = ctx.polar(a, 0.3, status=st, iters=20, prec="bf16")
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    del a
    if wide:
        y = y.T
    y = y.reshape(nb, n, n)
    bt = torch.from_numpy(b_tau / 32.0).cuda()                # FP64
    err2, ref2 = 0.0, 0.0
    tiles = []
    for k in range(0, nb, 128):  # FP64 error in slices of 128 blocks
        e = y[k:k + 128].double() - sgn[k:k + 128, :, None].double() * bt[None]
        err2 += float((e * e).sum())
        ref2 += 128 * float((bt * bt).sum())
        # squared error of every 128 x 128 tile of the output
        tiles.append((e * e).reshape(128, 8, 128, 8, 128).sum(dim=(2, 4)).flatten().cpu())
        del e
    rel = (err2 / ref2) ** 0.5
    t = torch.cat(tiles)
    spread = float((t.max() / t.mean()).sqrt())
    print(f"{'1024 x 2^20' if wide else '2^20 x 1024'} BF16 relerr {rel:.3e}, "
          f"128 x 128 tile spread {spread:.3f} over {t.numel()} tiles")
    assert rel < 2e-2
    assert spread < 2.0  # a partly wrong tile anywhere in 2^30 entries stands out


# --- guard bands (the stand-in for a memory checker) and the device-side timeout path

SENTINEL = 0x7FC0BEEF  # a NaN bit pattern that no kernel writes


def _gap(m, n, seed, tau=0.3):
    rng = np.random.default_rng(seed)
    k = min(m, n)
    lo = np.sort(rng.uniform(0.01, tau - 0.06, k // 2))
    hi = np.sort(rng.uniform(tau + 0.06, 1.0, k - k // 2 - 1))
    sig = np.sort(np.concatenate([lo, hi, [1.0]]))[::-1]
    import svt_workloads as wl
    return wl.spectrum_matrix(sig, m, n, seed)


def _guarded(m, n):
    """An m x n float view inside a larger buffer filled with SENTINEL, and the mask of
    the guard cells."""
    big = torch.full((m + 4, n + 12), SENTINEL, dtype=torch.int32, device="cuda")
    guard = torch.ones(big.shape, dtype=torch.bool, device="cuda")
    guard[2:2 + m, 5:5 + n] = False
    return big, big.view(torch.float32)[2:2 + m, 5:5 + n], guard


@pytest.mark.parametrize("m,n,prec", [(300, 200, "bf16"), (200, 300, "fp32"), (520, 130, "bf16")])
def test_guard_bands_around_output_and_workspace(m, n, prec):
    """Outputs written into views of larger sentinel-filled buffers, a sentinel tail after
    the workspace the solve sizes, the input compared before and after: every guard
    cell and the input are untouched, and the result is right."""
    a = _gap(m, n, m + n)
    exact = oracle.svt_definition(a.astype(np.float64), 0.3)
    need = pkg.workspace_bytes(m, n, iters=20, prec=prec)
    ctx = pkg.Context(0, workspace_bytes=need + (1 << 20))
    ctx.workspace[need:].fill_(0xA5)
    A = torch.from_numpy(a).cuda()
    A0 = A.clone()
    big, Y, guard = _guarded(m, n)
    ctx.polar(A, 0.3, out=Y, iters=20, prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(A, A0)
    assert bool((big[guard] == SENTINEL).all())
    assert bool((ctx.workspace[need:] == 0xA5).all())
    tol = 2e-2 if prec == "bf16" else 1e-4
    assert oracle.relerr(Y.cpu().numpy().astype(np.float64), exact) < tol


def test_guard_bands_around_batch_outputs():
    shapes = [(96, 64), (130, 260), (200, 200), (64, 128)]
    mats = [_gap(m, n, 7 + i) for i, (m, n) in enumerate(shapes)]
    ctx = pkg.Context(0, workspace_bytes=1 << 20)
    As = [torch.from_numpy(a).cuda() for a in mats]
    guarded = [_guarded(m, n) for m, n in shapes]
    ctx.batch(As, [0.3] * len(As), outs=[g[1] for g in guarded], opts={"iters": 20, "prec": "bf16"})
    torch.cuda.synchronize()
    for a, (big, Y, guard) in zip(mats, guarded):
        assert bool((big[guard] == SENTINEL).all())
        exact = oracle.svt_definition(a.astype(np.float64), 0.3)
        assert oracle.relerr(Y.cpu().numpy().astype(np.float64), exact) < 2e-2


def test_device_wait_timeout_is_reported_and_the_context_recovers():
    """A tile that waits for its own completion: the bounded wait runs out (~2 s), the
    kernel records SVT_ERR_TIMEOUT and returns without trapping, and later solves on
    the same context are correct."""
    import time
    ctx = pkg.Context(0, workspace_bytes=16 << 20)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.time()
    ctx.debug_wait_timeout(st)
    torch.cuda.synchronize()
    dt = time.time() - t0
    assert int(st.item()) == pkg.binding.ERR_TIMEOUT
    assert 1.5 < dt < 30, dt
    a = _gap(96, 64, 3)
    y = ctx.polar(torch.from_numpy(a).cuda(), 0.3, iters=20, prec="bf16")
    torch.cuda.synchronize()
    assert oracle.relerr(y.cpu().numpy().astype(np.float64),
                         oracle.svt_definition(a.astype(np.float64), 0.3)) < 2e-2
