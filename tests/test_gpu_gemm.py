"""Tensor-core product kernel (tcgen05 + TMA + TMEM) through the C ABI.

The reference is the exact product of the same BF16 inputs, formed in FP64 on
the host; the tolerance is the FP32-accumulation bound ~ K * 2^-24 relative to
sum |L||R|.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2607_22484_gb300")


@pytest.fixture(scope="module")
def ctx():
    return pkg.Context(0, workspace_bytes=1 << 20)


def _bf16(rows, cols, gen, ld=None):
    ld = ld or (cols + 7) // 8 * 8
    base = torch.zeros(rows, ld, dtype=torch.bfloat16, device="cuda")
    base[:, :cols] = (torch.randn(rows, cols, generator=gen) * 0.5).to(torch.bfloat16).cuda()
    return base[:, :cols]


def _check(D, exact, absmag, K):
    err = (D.double().cpu() - exact).abs()
    bound = 4 * K * 2.0 ** -24 * absmag + 1e-30
    ratio = (err / bound).max().item()
    assert ratio < 1.0, f"max err/bound = {ratio}"


# Tile-width codes: 0 automatic, 128 / 256 one CTA per tile, 512 a CTA pair per
# 256 x 256 tile (tcgen05 cta_group::2).
TILES = [0, 128, 256, 512]


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 256, 256), (300, 200, 130),
                                   (129, 257, 65), (64, 64, 64), (1000, 520, 777),
                                   (100, 300, 64), (513, 1030, 1100)])
def test_gemm_one_segment(ctx, M, N, K, tile):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    L = _bf16(M, K, g)
    R = _bf16(N, K, g)
    D = torch.full((M, N), float("nan"), device="cuda")
    ctx.debug_gemm_bf16(1, L, None, R, None, D, tile=tile)
    torch.cuda.synchronize()
    Ld, Rd = L.double().cpu(), R.double().cpu()
    _check(D, Ld @ Rd.T, Ld.abs() @ Rd.abs().T, K)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("N,K", [(256, 64), (520, 96), (1024, 300), (77, 40), (700, 130)])
def test_gemm_symmetric(ctx, N, K, tile):
    g = torch.Generator().manual_seed(N + K)
    L = _bf16(N, K, g)
    D = torch.full((N, N), float("nan"), device="cuda")
    ctx.debug_gemm_bf16(1, L, None, L, None, D, sym=True, tile=tile)
    torch.cuda.synchronize()
    Dc = D.cpu()
    assert torch.equal(Dc, Dc.T), "mirrored result must be bitwise symmetric"
    Ld = L.double().cpu()
    _check(D, Ld @ Ld.T, Ld.abs() @ Ld.abs().T, K)


def _split(x32):
    hi = x32.to(torch.bfloat16)
    lo = (x32 - hi.float()).to(torch.bfloat16)
    return hi, lo


@pytest.mark.parametrize("tile", [0, 512])
@pytest.mark.parametrize("nseg", [2, 3])
def test_gemm_split_segments(ctx, nseg, tile):
    """hi/lo splitting: 3 BF16 products reproduce an FP32 product to ~1e-5."""
    g = torch.Generator().manual_seed(nseg)
    M, N, K = 384, 320, 512
    L32 = torch.randn(M, K, generator=g).cuda()
    R32 = torch.randn(N, K, generator=g).cuda()
    Lh, Ll = _split(L32)
    Rh, Rl = _split(R32)
    D = torch.empty(M, N, device="cuda")
    ctx.debug_gemm_bf16(nseg, Lh, Ll, Rh, Rl, D, tile=tile)
    torch.cuda.synchronize()
    if nseg == 3:
        exact = L32.double().cpu() @ R32.double().cpu().T
        mag = L32.double().abs().cpu() @ R32.double().abs().cpu().T
        rel = ((D.double().cpu() - exact).abs() / mag).max().item()
        assert rel < 3e-5, rel
    else:
        exact = Lh.double().cpu() @ (Rh.double().cpu() + Rl.double().cpu()).T
        mag = Lh.double().abs().cpu() @ (Rh.double().abs().cpu() + Rl.double().abs().cpu()).T
        rel = ((D.double().cpu() - exact).abs() / mag).max().item()
        assert rel < 4 * K * 2.0 ** -24, rel


@pytest.mark.parametrize("tile", [0, 512])
def test_gemm_large_square(ctx, tile):
    """4096^3 product: samples of rows checked exactly (several waves of tiles)."""
    g = torch.Generator().manual_seed(4096)
    M = N = K = 4096
    L = (torch.randn(M, K, generator=g) * 0.1).to(torch.bfloat16).cuda()
    R = (torch.randn(N, K, generator=g) * 0.1).to(torch.bfloat16).cuda()
    D = torch.empty(M, N, device="cuda")
    ctx.debug_gemm_bf16(1, L, None, R, None, D, tile=tile)
    torch.cuda.synchronize()
    rows = torch.tensor([0, 1, 127, 128, 1000, 2047, 2048, 4000, 4095])
    Ls = L[rows.cuda()].double().cpu()
    Rd = R.double().cpu()
    _check(D[rows.cuda()], Ls @ Rd.T, Ls.abs() @ Rd.abs().T, K)
