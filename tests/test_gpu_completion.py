"""Matrix completion by proximal gradient through svt_prox_grad_step, against the
FP64 oracle loop (oracle/completion.py).

The instance is a scaled-down copy of the serving workload's completion client:
M = L R^T with L, R ~ N(0,1)^{256 x 5}, ||M||_2 ~ 10, a Bernoulli(0.2) mask.

* Gapped threshold: lambda halfway between sigma_5 and sigma_6 of P_Omega(M)
  (the signal / mask-noise gap, ~11 % of sigma_max). FP32 tier: relative error
  1e-4 of the result. BF16 tier: this threshold keeps 5 of 256 singular values,
  so ||A_tau||_F is ~15x smaller than ||Z||_F, while BF16 rounding acts on the
  operand (~2^-9 of ||Z||_F per product); the bound is therefore on the operand's
  scale, ||error||_F <= 8e-3 ||Z||_F (four units of 2^-9; one step measured
  4e-3 ||Z||_F, i.e. two units). The map
  X -> A_lambda(X + P_Omega(M - X)) is non-expansive (a gradient step of a
  1-smooth convex function with step 1, then a proximal operator), so T steps
  stay within T times the per-solve error of the oracle's iterate.
* The configured threshold lambda = 0.02 ||P_Omega(M)||_2 (no gap): the loop's
  objective and recovery error are compared with the oracle's.
* The device-resident loop (svt_complete: lambda continuation, relative-change
  stopping test, one graph launch): its iterates against the host loop and the
  oracle, its statistics against the oracle's stage rule, and the residual bound at
  its stop. With E the solve's error in the last step (FP32 tier: <= 1e-4 of the
  result here), ||P_Omega(M - X)||_2 <= lambda + (1 + 1/h) ||X - X_prev||_F + ||E||_F / h;
  the relative change is ||X - X_prev||_F / ||P_Omega(M)||_F.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import completion as oc
import svt_workloads as wl

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2607_22484_gb300")

N, RANK = 256, 5


@pytest.fixture(scope="module")
def ctx():
    return pkg.Context(0, workspace_bytes=64 << 20)


@pytest.fixture(scope="module")
def inst():
    m, mask = wl.completion_problem(N, RANK)
    m64 = m.astype(np.float64)
    pm = np.where(mask != 0, m64, 0.0)
    s = np.linalg.svd(pm, compute_uv=False)
    return m, mask.astype(np.uint8), 0.5 * (s[RANK - 1] + s[RANK]), 0.02 * s[0]


def _dev(m, mask):
    return torch.from_numpy(m).cuda(), torch.from_numpy(mask).cuda()


def _bound(prec, result, operand):
    """Allowed Frobenius error of one solve: relative to the result (FP32 tier) or
    to the operand's scale (BF16 tier), see the module docstring."""
    if prec == "fp32":
        return 1e-4 * np.linalg.norm(result)
    return 8e-3 * np.linalg.norm(operand)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_one_step_gapped(ctx, inst, prec):
    m, mask, lam_gap, _ = inst
    x0 = (np.random.default_rng(3).standard_normal(m.shape) * 0.01).astype(np.float32)
    M, W = _dev(m, mask)
    X = torch.from_numpy(x0.copy()).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.prox_grad_step(X, M, W, lam_gap, status=status, iters=20, prec=prec)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    x64, m64 = x0.astype(np.float64), m.astype(np.float64)
    ref = oc.prox_grad_step(x64, m64, mask, lam_gap)
    z = np.where(mask != 0, m64, x64)
    err = np.linalg.norm(X.cpu().numpy().astype(np.float64) - ref)
    print(f"{prec}: one step, relerr {err / np.linalg.norm(ref):.2e}, "
          f"error / ||Z||_F {err / np.linalg.norm(z):.2e}")
    assert err < _bound(prec, ref, z), err


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_loop_gapped(ctx, inst, prec):
    m, mask, lam_gap, _ = inst
    steps = 10
    M, W = _dev(m, mask)
    X = ctx.complete(M, W, lam_gap, steps, iters=20, prec=prec)
    torch.cuda.synchronize()
    m64 = m.astype(np.float64)
    ref, x = None, np.zeros_like(m64)
    bound = 0.0
    for _ in range(steps):  # oracle iterates, and the per-step bounds along them
        z = np.where(mask != 0, m64, x)
        x = oc.prox_grad_step(x, m64, mask, lam_gap)
        bound += _bound(prec, x, z)
    ref = x
    err = np.linalg.norm(X.cpu().numpy().astype(np.float64) - ref)
    rec_gpu = np.linalg.norm(X.cpu().numpy() - m) / np.linalg.norm(m)
    rec_ref = np.linalg.norm(ref - m) / np.linalg.norm(m)
    print(f"{prec}: iterate error {err:.2e} (bound {bound:.2e}), recovery {rec_gpu:.4f} "
          f"(oracle {rec_ref:.4f})")
    assert err < bound, (err, bound)


def test_loop_configured_lambda_fp32(ctx, inst):
    """lambda = 0.02 ||P_Omega(M)||_2: no gap at the threshold; the loop's objective
    and recovery error follow the oracle's."""
    m, mask, _, lam = inst
    steps = 8
    M, W = _dev(m, mask)
    X = ctx.complete(M, W, lam, steps, iters=20, prec="fp32")
    torch.cuda.synchronize()
    ref = oc.complete(m, mask, lam, steps)
    x = X.cpu().numpy().astype(np.float64)
    f_gpu = oc.objective(x, m.astype(np.float64), mask, lam)
    f_ref = oc.objective(ref, m.astype(np.float64), mask, lam)
    assert abs(f_gpu - f_ref) < 1e-3 * f_ref, (f_gpu, f_ref)
    rec_gpu = np.linalg.norm(x - m) / np.linalg.norm(m)
    rec_ref = np.linalg.norm(ref - m) / np.linalg.norm(m)
    assert abs(rec_gpu - rec_ref) < 1e-3, (rec_gpu, rec_ref)


def test_strided_buffers_match_contiguous(ctx, inst):
    """Row pitches that break 16-byte alignment take the scalar path of the masked
    update; the result equals the contiguous one."""
    m, mask, lam_gap, _ = inst
    M, W = _dev(m, mask)
    X1 = ctx.complete(M, W, lam_gap, 2, iters=20, prec="fp32")
    Mb = torch.zeros(N, N + 5, device="cuda")
    Mb[:, 1:N + 1] = M
    Wb = torch.zeros(N, N + 3, dtype=torch.uint8, device="cuda")
    Wb[:, 2:N + 2] = W
    Xb = torch.zeros(N, N + 7, device="cuda")
    Zb = torch.empty(N, N + 1, device="cuda")
    Ms, Ws, Xs, Zs = Mb[:, 1:N + 1], Wb[:, 2:N + 2], Xb[:, 3:N + 3], Zb[:, :N]
    for _ in range(2):
        ctx.prox_grad_step(Xs, Ms, Ws, lam_gap, Z=Zs, iters=20, prec="fp32")
    torch.cuda.synchronize()
    assert oracle.relerr(Xs.cpu().numpy().astype(np.float64),
                         X1.cpu().numpy().astype(np.float64)) < 1e-5


def test_invalid_arguments(ctx, inst):
    m, mask, lam_gap, _ = inst
    M, W = _dev(m, mask)
    X = torch.zeros_like(M)
    with pytest.raises(pkg.SVTError):
        ctx.prox_grad_step(X, M, W, lam_gap, Z=X)          # Z aliases X
    with pytest.raises(pkg.SVTError):
        ctx.prox_grad_step(X, M, W, lam_gap, Z=M.clone(), step=0.0)
    with pytest.raises(pkg.SVTError):
        ctx.prox_grad_step(X, M, W, -1.0)
    with pytest.raises(pkg.SVTError):
        ctx.prox_grad_step(X, M, W, float("inf"))
    with pytest.raises(ValueError):
        ctx.prox_grad_step(X, M, W.float(), lam_gap)     # mask must be bytes


# --- the device-resident loop (svt_complete)

def _stats(st):
    return pkg.read_completion_stats(st)


def test_device_loop_fixed_steps_matches_host_loop(ctx, inst):
    """One stage, tol 0: the loop runs max_steps steps of the same step as the host
    loop of svt_prox_grad_step."""
    m, mask, lam_gap, _ = inst
    M, W = _dev(m, mask)
    before = ctx.launch_count()
    X, st = ctx.complete_on_device(M, W, lam_gap, 6, iters=20, prec="fp32")
    assert ctx.launch_count() == before + 1
    s = _stats(st)
    assert (s["steps"], s["stages"], s["stage_steps"], s["status"]) == (6, 1, 6, 0)
    assert s["lam"] == pytest.approx(lam_gap, rel=1e-6)
    Xh = ctx.complete(M, W, lam_gap, 6, iters=20, prec="fp32")
    torch.cuda.synchronize()
    assert oracle.relerr(X.cpu().numpy().astype(np.float64),
                         Xh.cpu().numpy().astype(np.float64)) < 1e-5
    # the last relative change is the one of the iterates
    x5 = ctx.complete(M, W, lam_gap, 5, iters=20, prec="fp32").cpu().numpy().astype(np.float64)
    x6 = X.cpu().numpy().astype(np.float64)
    scale = np.linalg.norm(np.where(mask != 0, m.astype(np.float64), 0.0))
    assert s["data_norm"] == pytest.approx(scale, rel=1e-12)
    rho = np.linalg.norm(x6 - x5) / scale
    assert abs(s["rel_change"] - rho) < 0.05 * rho + 2e-6, (s["rel_change"], rho)


def test_device_loop_continuation_against_the_oracle(ctx, inst):
    """Continuation from 2.5 times the gapped lambda down to it, tol 1e-4: same stage
    count as the oracle's rule, the stop's residual bound, and the oracle's minimum."""
    m, mask, lam_gap, _ = inst
    m64 = m.astype(np.float64)
    lam0, eta, tol, cap = 2.5 * lam_gap, 0.5, 1e-4, 8
    M, W = _dev(m, mask)
    X, st = ctx.complete_on_device(M, W, lam_gap, 120, lam0=lam0, eta=eta, tol=tol,
                                   stage_steps=cap, iters=20, prec="fp32")
    s = _stats(st)
    x = X.cpu().numpy().astype(np.float64)
    xo, info = oc.complete_continuation(m64, mask, lam_gap, lam0, eta, tol, 120, stage_steps=cap)
    print(f"device loop: {s}; oracle: steps {info['steps']}, stages {info['stages']}, "
          f"rho {info['rel_change']:.2e}")
    assert s["status"] == 0
    assert s["stages"] == info["stages"]
    assert s["lam"] == pytest.approx(lam_gap, rel=1e-6)
    assert s["steps"] < 120 and s["rel_change"] <= tol
    assert abs(s["steps"] - info["steps"]) <= 4, (s["steps"], info["steps"])
    g = np.where(mask != 0, m64 - x, 0.0)
    r = s["rel_change"] * s["data_norm"]
    bound = lam_gap + 2.0 * r + 1e-4 * np.linalg.norm(x)
    assert np.linalg.norm(g, 2) <= bound, (np.linalg.norm(g, 2), bound)
    f_gpu = oc.objective(x, m64, mask, lam_gap)
    f_ref = oc.objective(xo, m64, mask, lam_gap)
    assert abs(f_gpu - f_ref) < 1e-4 * f_ref, (f_gpu, f_ref)


def test_device_loop_stage_caps(ctx, inst):
    """tol 0 and a cap of 2 steps per stage: 2 + 2 + the rest in the last stage (the
    stage lambdas stay below sigma_max of P_Omega(M), so no stage's iterate stays
    exactly put, which would end it at tol 0)."""
    m, mask, lam_gap, _ = inst
    M, W = _dev(m, mask)
    _, st = ctx.complete_on_device(M, W, lam_gap, 9, lam0=1.4 * lam_gap, eta=0.8,
                                   stage_steps=2, iters=12, prec="bf16")
    s = _stats(st)
    assert (s["steps"], s["stages"], s["stage_steps"], s["status"]) == (9, 3, 5, 0)
    _, info = oc.complete_continuation(m.astype(np.float64), mask, lam_gap, 1.4 * lam_gap, 0.8,
                                       0.0, 9, stage_steps=2)
    assert [info["stage_of_step"].count(k) for k in range(3)] == [2, 2, 5]


def test_device_loop_bf16_against_the_oracle(ctx, inst):
    """BF16 tier, one stage, 10 steps: within the per-step operand-scale bound of the
    oracle's iterates (as the host loop)."""
    m, mask, lam_gap, _ = inst
    M, W = _dev(m, mask)
    X, st = ctx.complete_on_device(M, W, lam_gap, 10, iters=20, prec="bf16")
    s = _stats(st)
    assert (s["steps"], s["status"]) == (10, 0)
    m64 = m.astype(np.float64)
    x, bound = np.zeros_like(m64), 0.0
    for _ in range(10):
        z = np.where(mask != 0, m64, x)
        x = oc.prox_grad_step(x, m64, mask, lam_gap)
        bound += _bound("bf16", x, z)
    err = np.linalg.norm(X.cpu().numpy().astype(np.float64) - x)
    assert err < bound, (err, bound)


def test_device_loop_zero_steps_and_relaunch(ctx, inst):
    m, mask, lam_gap, _ = inst
    M, W = _dev(m, mask)
    x0 = torch.from_numpy(
        (np.random.default_rng(5).standard_normal(m.shape) * 0.01).astype(np.float32)).cuda()
    X = x0.clone()
    _, st = ctx.complete_on_device(M, W, lam_gap, 0, X=X, iters=20, prec="fp32")
    s = _stats(st)
    assert (s["steps"], s["stages"], s["status"]) == (0, 0, 0)
    assert torch.equal(X, x0)
    # the same arguments twice: the cached graph runs again from the reset start
    Z = torch.empty_like(M)
    P = torch.empty_like(M)
    outs = []
    for _ in range(2):
        X.copy_(x0)
        ctx.complete_on_device(M, W, lam_gap, 4, X=X, Z=Z, Xprev=P, stats=st, iters=20,
                               prec="fp32")
        outs.append(X.clone())
        assert _stats(st)["steps"] == 4
    assert oracle.relerr(outs[0].cpu().numpy().astype(np.float64),
                         outs[1].cpu().numpy().astype(np.float64)) < 1e-6


def test_device_loop_stops_on_a_nonfinite_solve(ctx, inst):
    m, mask, lam_gap, _ = inst
    mm = m.copy()
    i, j = np.argwhere(mask != 0)[0]
    mm[i, j] = np.nan
    M, W = _dev(mm, mask)
    _, st = ctx.complete_on_device(M, W, lam_gap, 5, iters=8, prec="bf16")
    s = _stats(st)
    assert s["status"] == pkg.binding.ERR_NONFINITE
    assert s["steps"] == 1


def test_device_loop_invalid_arguments(ctx, inst):
    m, mask, lam_gap, _ = inst
    M, W = _dev(m, mask)
    X = torch.zeros_like(M)
    bad = [
        dict(lam0=0.5 * lam_gap),                 # lam0 < lam
        dict(lam0=2 * lam_gap, eta=1.0),          # no decrease
        dict(lam0=2 * lam_gap, eta=0.0),
        dict(tol=-1.0),
        dict(stage_steps=-1),
        dict(step=0.0),
    ]
    for kw in bad:
        with pytest.raises(pkg.SVTError):
            ctx.complete_on_device(M, W, lam_gap, 3, X=X, **kw)
    with pytest.raises(pkg.SVTError):                 # more than 64 stages
        ctx.complete_on_device(M, W, 0.0, 3, lam0=1.0, eta=0.5, X=X)
    with pytest.raises(pkg.SVTError):                 # negative step count
        ctx.complete_on_device(M, W, lam_gap, -1, X=X)
    with pytest.raises(pkg.SVTError):                 # Xprev aliases X
        ctx.complete_on_device(M, W, lam_gap, 3, X=X, Xprev=X)
    st = torch.zeros(pkg.binding.COMPLETION_STATS_BYTES + 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):                   # misaligned statistics
        ctx.complete_on_device(M, W, lam_gap, 3, X=X, stats=st[1:])
