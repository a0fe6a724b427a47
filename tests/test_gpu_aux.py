"""Auxiliary subsystems through the C ABI: host-side fault injection (a failing plan
build, a serving admission delay, a device dependency-wait limit that runs out),
serving cancellation, per-request JSONL records, and the autotune cache kept as
JSON across contexts. Every injected failure is an ordinary error status: nothing
here makes the GPU fault, trap or hang."""
import json
import time

import numpy as np
import pytest
import torch

import oracle
import svt_workloads as wl

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2607_22484_gb300")
B = pkg.binding


def _gap_matrix(m, n, seed, tau=0.3):
    k = min(m, n)
    rng = np.random.default_rng(seed)
    lo = np.sort(rng.uniform(0.01, tau - 0.06, k // 2))
    hi = np.sort(rng.uniform(tau + 0.06, 1.0, k - k // 2 - 1))
    sig = np.sort(np.concatenate([lo, hi, [1.0]]))[::-1]
    return wl.spectrum_matrix(sig, m, n, seed)


def _wait(ctx, tickets, limit_s=120):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets) and time.time() - t0 < limit_s:
        for t in tickets:
            if t not in res:
                st, lat = ctx.poll(t)
                if st != B.ERR_NOT_READY:
                    res[t] = (st, lat)
        time.sleep(0.001)
    assert len(res) == len(tickets), "serving did not finish"
    return res


def test_failing_plan_build_is_reported_and_the_next_call_works():
    ctx = pkg.Context(0, workspace_bytes=64 << 20)
    a = _gap_matrix(200, 150, seed=1)
    dev = torch.from_numpy(a).cuda()
    ctx.debug("fail_plan", 1)
    with pytest.raises(pkg.SVTError) as e:
        ctx.polar(dev, 0.3, iters=20, prec="bf16")
    assert e.value.status == B.ERR_OOM
    y = ctx.polar(dev, 0.3, iters=20, prec="bf16")  # the counter is spent: builds again
    torch.cuda.synchronize()
    exact = oracle.svt_definition(a.astype(np.float64), 0.3)
    assert oracle.relerr(y.cpu().numpy(), exact) < 2e-2
    with pytest.raises(pkg.SVTError):
        ctx.debug("fail_plan", -1)


def test_failing_plan_build_fails_one_serving_request_only():
    ctx = pkg.Context(0, workspace_bytes=256 << 20)
    shapes = [(160, 120), (176, 136), (192, 150)]
    mats = [torch.from_numpy(_gap_matrix(m, n, seed=m)).cuda() for m, n in shapes]
    outs = [torch.full_like(a, float("nan")) for a in mats]
    torch.cuda.synchronize()
    ctx.debug("fail_plan", 2)  # the second admission's plan build fails
    tickets = [ctx.submit(a, 0.3, y, iters=20, prec="bf16") for a, y in zip(mats, outs)]
    res = _wait(ctx, tickets)
    sts = [res[t][0] for t in tickets]
    assert sts == [B.OK, B.ERR_OOM, B.OK], sts
    for i in (0, 2):
        exact = oracle.svt_definition(mats[i].cpu().numpy().astype(np.float64), 0.3)
        assert oracle.relerr(outs[i].cpu().numpy(), exact) < 2e-2
    for t in tickets:
        assert ctx.release(t) == B.OK


def test_dependency_wait_limit_runs_out_and_the_context_recovers():
    """A wait limit of 1 ns makes the fused launch's first unmet dependency wait give
    up: the solve reports SVT_ERR_TIMEOUT through its status word (the kernel drains
    its copies and MMAs and frees tensor memory), and with the default limit restored
    the same context solves correctly."""
    ctx = pkg.Context(0, workspace_bytes=pkg.workspace_bytes(1024, 768, prec="bf16"))
    a = _gap_matrix(1024, 768, seed=5)
    dev = torch.from_numpy(a).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.debug("wait_limit_ns", 1)
    ctx.polar(dev, 0.3, status=st, iters=20, prec="bf16", tile=256)
    torch.cuda.synchronize()
    assert int(st.item()) == B.ERR_TIMEOUT
    ctx.debug("wait_limit_ns", 0)
    st.zero_()
    y = ctx.polar(dev, 0.3, status=st, iters=20, prec="bf16", tile=256)
    torch.cuda.synchronize()
    assert int(st.item()) == B.OK
    exact = oracle.svt_definition(a.astype(np.float64), 0.3)
    assert oracle.relerr(y.cpu().numpy(), exact) < 2e-2


def test_admission_delay_holds_requests():
    ctx = pkg.Context(0, workspace_bytes=256 << 20)
    mats = [torch.from_numpy(_gap_matrix(128 + 16 * i, 96, seed=20 + i)).cuda() for i in range(3)]
    outs = [torch.empty_like(a) for a in mats]
    torch.cuda.synchronize()
    ctx.debug("admit_delay_us", 40000)
    tickets = [ctx.submit(a, 0.3, y, iters=20, prec="bf16") for a, y in zip(mats, outs)]
    res = _wait(ctx, tickets)
    for t, a, y in zip(tickets, mats, outs):
        st, lat = res[t]
        assert st == B.OK and lat >= 40.0, (st, lat)
        exact = oracle.svt_definition(a.cpu().numpy().astype(np.float64), 0.3)
        assert oracle.relerr(y.cpu().numpy(), exact) < 2e-2
    ctx.debug("admit_delay_us", 0)


def test_cancel_queued_and_running_requests(tmp_path):
    """Cancelling a queued request removes it (it polls SVT_ERR_CANCELLED and leaves
    no record of work); cancelling a request whose stages are being issued either drops
    it (OK, then CANCELLED) or finds its last stage already out (ERR_BUSY, then its
    normal result); the others complete as if alone; JSONL records cover every
    retired request with its status."""
    log = tmp_path / "serve.jsonl"
    ctx = pkg.Context(0, workspace_bytes=512 << 20)
    ctx.serve_metrics(log)
    mats = [torch.from_numpy(_gap_matrix(200 + 8 * i, 160, seed=40 + i)).cuda() for i in range(5)]
    big = torch.from_numpy(_gap_matrix(2048, 1536, seed=49)).cuda()  # small lane, many windows
    outs = [torch.empty_like(a) for a in mats]
    ybig = torch.empty_like(big)
    torch.cuda.synchronize()
    ctx.debug("admit_delay_us", 200000)  # everything stays queued for 200 ms
    tickets = [ctx.submit(a, 0.3, y, iters=20, prec="bf16") for a, y in zip(mats, outs)]
    assert ctx.cancel(tickets[1]) == B.OK
    assert ctx.cancel(tickets[3]) == B.OK
    assert ctx.poll(tickets[1])[0] == B.ERR_CANCELLED
    ctx.debug("admit_delay_us", 0)
    tb = ctx.submit(big, 0.3, ybig, iters=20, prec="bf16")
    time.sleep(0.003)  # admitted by now, its windows going out one stage at a time
    rc = ctx.cancel(tb)
    res = _wait(ctx, tickets + [tb])
    assert res[tickets[1]][0] == B.ERR_CANCELLED and res[tickets[3]][0] == B.ERR_CANCELLED
    alone = pkg.Context(0, workspace_bytes=64 << 20)
    for i in (0, 2, 4):
        assert res[tickets[i]][0] == B.OK
        ref = alone.polar(mats[i], 0.3, iters=20, prec="bf16")
        torch.cuda.synchronize()
        assert oracle.relerr(outs[i].cpu().numpy(), ref.cpu().numpy()) < 1e-5
    if rc == B.OK:  # dropped before a later window (or still queued)
        assert res[tb][0] == B.ERR_CANCELLED
    else:  # its last stage was already out (BUSY) or it had finished (INVALID)
        assert rc in (B.ERR_BUSY, B.ERR_INVALID) and res[tb][0] == B.OK
    print(f"cancel of a running 2048 x 1536 request after 3 ms: {pkg.status_str(rc)}")
    assert ctx.cancel(tickets[0]) == B.ERR_INVALID  # completed
    assert ctx.cancel(123456789) == B.ERR_INVALID    # unknown
    # the context keeps serving
    t2 = ctx.submit(mats[0], 0.3, outs[0], iters=20, prec="bf16")
    assert _wait(ctx, [t2])[t2][0] == B.OK
    ctx.serve_metrics(None)
    recs = [json.loads(line) for line in log.read_text().splitlines()]
    by = {r["ticket"]: r for r in recs}
    for t in tickets + [tb, t2]:
        st = res[t][0] if t in res else B.OK
        assert by[t]["status"] == pkg.status_str(st), (t, by[t])
        assert by[t]["lane"] == "small" and by[t]["prec"] == "bf16" and by[t]["iters"] == 20
        assert by[t]["latency_ms"] >= by[t]["queue_ms"] >= 0.0
    assert abs(by[tickets[0]]["latency_ms"] - res[tickets[0]][1]) < 1.0
    assert by[tickets[1]]["run_ms"] == 0.0  # never admitted


def test_tuning_cache_roundtrip_and_gpu_key():
    a = torch.from_numpy(_gap_matrix(640, 512, seed=21)).cuda()
    ctx = pkg.Context(0, workspace_bytes=1 << 20)
    ctx.autotune(a, 0.3, iters=20, prec="bf16")
    text = ctx.tuning_export()
    doc = json.loads(text)
    assert doc["format"] == 1 and doc["gpu"] == torch.cuda.get_device_name(0)
    assert doc["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    (e,) = [e for e in doc["entries"] if (e["m"], e["n"]) == (640, 512)]
    assert e["prec"] == B.BF16 and e["iters"] == 20 and all(w in (128, 256, 512) for w in e["widths"])
    # a fresh context imports it and solves with the same plan (same result)
    y0 = ctx.polar(a, 0.3, iters=20, prec="bf16")
    other = pkg.Context(0, workspace_bytes=1 << 20)
    other.tuning_import(text)
    assert json.loads(other.tuning_export()) == doc
    y1 = other.polar(a, 0.3, iters=20, prec="bf16")
    torch.cuda.synchronize()
    assert oracle.relerr(y1.cpu().numpy(), y0.cpu().numpy()) < 1e-5
    # growing the workspace keeps the tuning
    other.ensure_workspace(other.workspace.numel() * 4)
    assert json.loads(other.tuning_export()) == doc
    # tuned on another GPU, or not JSON of this format: rejected, nothing imported
    fresh = pkg.Context(0, workspace_bytes=1 << 20)
    for bad in (text.replace(doc["gpu"], doc["gpu"] + " X"),
                text.replace(f'"sms": {doc["sms"]}', f'"sms": {doc["sms"] + 1}'),
                text.replace('"format": 1', '"format": 2'), text[:-5], "[]",
                text.replace('"widths": [', '"widths": [300, ')):
        with pytest.raises(pkg.SVTError) as err:
            fresh.tuning_import(bad)
        assert err.value.status == B.ERR_INVALID
    assert json.loads(fresh.tuning_export())["entries"] == []


def test_large_lane_alone_and_cancel_between_launches(tmp_path):
    """A large request (at least 8 Mi elements) is issued as consecutive fused launches
    over parts of its product table: alone it runs them on every SM and equals the same
    solve through svt_polar; cancelled while its launches are being issued it stops
    before the next one and polls SVT_ERR_CANCELLED (or, were it already fully issued,
    the cancel answers SVT_ERR_BUSY and the result is normal), and the context keeps
    serving."""
    log = tmp_path / "large.jsonl"
    ctx = pkg.Context(0, workspace_bytes=pkg.workspace_bytes(8192, 4096, prec="fp32") + (256 << 20))
    ctx.serve_metrics(log)
    a = torch.from_numpy(_gap_matrix(4096, 2048, seed=61)).cuda()
    y = torch.full_like(a, float("nan"))
    torch.cuda.synchronize()
    for _ in range(2):  # the first submission builds the plan
        t = ctx.submit(a, 0.3, y, iters=20, prec="bf16")
        assert _wait(ctx, [t])[t][0] == B.OK
        assert ctx.release(t) == B.OK
    ref = pkg.Context(0, workspace_bytes=1 << 20).polar(a, 0.3, iters=20, prec="bf16")
    torch.cuda.synchronize()
    assert oracle.relerr(y.cpu().numpy(), ref.cpu().numpy()) < 1e-5

    big = torch.from_numpy(_gap_matrix(8192, 4096, seed=62)).cuda()
    ybig = torch.empty_like(big)
    small = torch.from_numpy(_gap_matrix(256, 192, seed=63)).cuda()
    ysmall = torch.empty_like(small)
    torch.cuda.synchronize()
    tb = ctx.submit(big, 0.3, ybig, iters=20, prec="fp32")  # about 100 ms of launches
    time.sleep(0.02)
    rc = ctx.cancel(tb)
    res = _wait(ctx, [tb])
    if rc == B.OK:
        assert res[tb][0] == B.ERR_CANCELLED
    else:
        assert rc == B.ERR_BUSY and res[tb][0] == B.OK
    print(f"cancel of a running 8192 x 4096 FP32-tier request after 20 ms: {pkg.status_str(rc)}")
    ts = ctx.submit(small, 0.3, ysmall, iters=20, prec="bf16")
    assert _wait(ctx, [ts])[ts][0] == B.OK
    exact = oracle.svt_definition(small.cpu().numpy().astype(np.float64), 0.3)
    assert oracle.relerr(ysmall.cpu().numpy(), exact) < 2e-2
    ctx.serve_metrics(None)
    recs = {r["ticket"]: r for r in map(json.loads, log.read_text().splitlines())}
    assert recs[tb]["lane"] == "large" and recs[ts]["lane"] == "small"
    assert recs[tb]["status"] == pkg.status_str(res[tb][0])
