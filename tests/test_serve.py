"""Request server: continuous batching with HBM admission (needs a GB300).

Each request's result must be the same alone and in the mix (tolerance: 0
bytes), equal to the direct C-ABI result, and the admission must respect the
budget while still batching concurrent requests (a request that finds the
server idle is launched on the submitting thread at once).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z

pytestmark = pytest.mark.gpu


def _requests():
    rng = np.random.default_rng(40)
    reqs = []
    for i in range(36):
        dt = ["bf16", "fp16", "fp32"][i % 3]
        es = {"bf16": 2, "fp16": 2, "fp32": 4}[dt]
        nbytes = int(np.exp(rng.uniform(np.log(64 << 10), np.log(6 << 20)))) // es * es
        n = nbytes // es
        x = W.gaussian(n, 0.02, 1000 + i, W.TORCH_DTYPE[dt], device="cuda")
        delta = (i % 7 == 3)
        base = None
        if delta:
            base = (x.float() + 1e-4 * torch.randn(n, device="cuda")).to(x.dtype)
        op = "decompress" if i % 3 == 1 else "compress"
        reqs.append((op, x, base))
    return reqs


def _collect(server: Z.Server, results: dict, want: int, timeout_s: float = 120.0):
    """Poll completions, copy each output out and release it (releasing frees
    budget for queued requests) until `want` results are in."""
    import time
    t_end = time.time() + timeout_s
    while len(results) < want:
        assert time.time() < t_end, "server did not finish"
        for c in server.poll():
            assert c.status == 0
            assert c.t_submit <= c.t_admit <= c.t_done
            results[c.tag] = server.output(c).cpu().numpy().tobytes()
            server.release(c.id)
        time.sleep(0.001)


def _run(server: Z.Server, reqs, containers, one_at_a_time: bool):
    results = {}
    for i, (op, x, base) in enumerate(reqs):
        if op == "compress":
            server.submit_compress(x, base=base, tag=i)
        else:
            server.submit_decompress(containers[i], base=base, tag=i)
        if one_at_a_time:
            _collect(server, results, i + 1)
    _collect(server, results, len(reqs))
    return results


def test_results_identical_alone_and_in_the_mix():
    torch.cuda.set_device(0)
    reqs = _requests()
    containers = {}
    for i, (op, x, base) in enumerate(reqs):
        if op == "decompress":
            containers[i] = Z.compress(x, base=base)
    alone = Z.Server(1 << 30, slots=1)
    r_alone = _run(alone, reqs, containers, one_at_a_time=True)
    alone.close()
    # small budget: forces queueing and admission; 4 slots: overlapping batches
    mix = Z.Server(48 << 20, slots=4)
    r_mix = _run(mix, reqs, containers, one_at_a_time=False)
    st = mix.stats()
    mix.close()
    assert set(r_alone) == set(r_mix) == set(range(len(reqs)))
    for i in range(len(reqs)):
        assert r_alone[i] == r_mix[i], i
    assert st.completed == len(reqs)
    # one slot and room for all: a request submitted to an idle server is
    # launched at once, the ones arriving while it runs queue and go out
    # together as one batch
    one = Z.Server(1 << 30, slots=1)
    r_one = _run(one, reqs, containers, one_at_a_time=False)
    st1 = one.stats()
    one.close()
    assert r_one == r_alone
    assert st1.completed == len(reqs) and st1.max_batch > 1
    # the results are the codec's: containers equal the direct API's (and the
    # oracle's for a sample), decoded tensors equal their inputs
    for i, (op, x, base) in enumerate(reqs):
        xb = x.contiguous().view(torch.uint8).cpu().numpy()
        if op == "compress":
            assert r_mix[i] == Z.compress(x, base=base).to_bytes()
            if i % 6 == 0:
                code = Z.dtype_code(x, None)
                if base is None:
                    want = O.compress(xb, code, Z.DEFAULT_CHUNK)
                else:
                    want = O.delta(xb, base.contiguous().view(torch.uint8).cpu().numpy(), code,
                                   Z.DEFAULT_CHUNK)
                assert r_mix[i] == want
        else:
            assert r_mix[i] == xb.tobytes()


def test_admission_refuses_what_can_never_fit():
    s = Z.Server(4 << 20, slots=2)
    x = torch.zeros(4 << 20, dtype=torch.bfloat16, device="cuda")   # 8 MiB > budget
    with pytest.raises(Z.ZipnnError) as e:
        s.submit_compress(x)
    assert e.value.status == -6
    s.close()


def test_budget_is_respected_under_a_burst():
    s = Z.Server(24 << 20, slots=4)
    xs = [W.gaussian(1 << 20, 0.02, 2000 + i, device="cuda") for i in range(24)]  # 2 MiB each
    ids = [s.submit_compress(x, tag=i) for i, x in enumerate(xs)]
    peak = 0
    done = []
    while len(done) < len(ids):
        st = s.stats()
        peak = max(peak, st.arena_used + st.inputs_charged)
        for c in s.poll():
            done.append(c)
            s.release(c.id)
    assert peak <= 24 << 20
    for c in done:
        assert c.status == 0
    s.close()


def test_corrupt_container_fails_its_request_and_the_server_goes_on():
    """Each batch's kernels report into the batch's own device error word: a
    container whose map entry names no valid mode completes with ECORRUPT,
    and the next request (same slot) completes normally."""
    import time
    x = W.gaussian(300_000, 0.02, 3000, device="cuda")
    c = Z.compress(x)
    buf = c.device_tensor().clone()
    buf[64 + 12] = 7                                    # invalid mode in the first map entry
    bad = Z.wrap(buf)
    s = Z.Server(1 << 28, slots=1)
    got = {}
    for tag, cont in ((0, bad), (1, c)):
        s.submit_decompress(cont, tag=tag)
        t_end = time.time() + 60
        while tag not in got:
            assert time.time() < t_end, "server did not finish"
            for comp in s.poll():
                got[comp.tag] = (comp.status, s.output(comp).cpu().numpy().tobytes()
                                 if comp.status == 0 else None)
                s.release(comp.id)
            time.sleep(0.001)
    s.close()
    assert got[0][0] == -3                               # ZIPNN_ECORRUPT
    assert got[1][0] == 0
    assert got[1][1] == x.view(torch.uint8).cpu().numpy().tobytes()
    # the library's own error word was not touched
    Z.sync_status()


def test_batch_workspace_that_does_not_fit_hands_back_the_tail():
    """Two compress requests whose inputs and outputs fit the budget together,
    but whose combined encoder workspace does not: the admission pass that
    takes both must hand the second back (arrival order kept) and run the
    first alone, and both must complete.  A decompress request's output, held
    until released, keeps both queued so that one pass sees them together."""
    import ctypes
    import time
    torch.cuda.set_device(0)
    chunk = Z.DEFAULT_CHUNK
    n = 16 << 20                                  # elements: 32 MiB of BF16 each
    nb = 2 * n
    a256 = lambda v: (v + 255) // 256 * 256

    def batch_ws(k):
        sizes = (ctypes.c_size_t * k)(*([nb] * k))
        dts = (ctypes.c_int * k)(*([Z.BF16] * k))
        return int(Z.lib().zipnn_batch_compress_workspace_size(sizes, dts, k, chunk))

    out = a256(Z.compress_bound(nb, Z.BF16, chunk))
    ws1, ws2 = batch_ws(1), batch_ws(2)
    assert ws2 - ws1 > 8192
    budget = 2 * nb + 2 * out + ws2 - 4096        # both fit, their joint workspace does not
    assert nb + out + ws1 <= budget               # the first alone does
    x1 = W.gaussian(n, 0.02, 3100, device="cuda")
    x2 = W.gaussian(n, 0.02, 3101, device="cuda")
    # the blocker's output (held) leaves no room for the first compress request
    n0 = (budget - nb - out) // 2 + (1 << 20)
    x0 = W.gaussian(n0, 0.02, 3102, device="cuda")
    c0 = Z.compress(x0)
    assert c0.nbytes + a256(2 * n0) <= budget
    s = Z.Server(budget, slots=1)
    id0 = s.submit_decompress(c0, tag=0)
    got, t_end = {}, time.time() + 60
    while 0 not in got:
        assert time.time() < t_end, "server did not finish"
        for c in s.poll():
            got[c.tag] = c
        time.sleep(0.001)
    assert got[0].status == 0
    s.submit_compress(x1, tag=1)
    s.submit_compress(x2, tag=2)
    time.sleep(0.05)
    assert s.poll() == []                         # both wait for the blocker's memory
    s.release(id0)
    res, t_end = {}, time.time() + 60
    while len(res) < 2:
        assert time.time() < t_end, "server did not finish"
        for c in s.poll():
            assert c.status == 0, (c.tag, c.status)
            res[c.tag] = s.output(c).cpu().numpy().tobytes()
            s.release(c.id)
        time.sleep(0.001)
    st = s.stats()
    s.close()
    assert st.max_batch == 1                      # the joint batch was split
    assert res[1] == Z.compress(x1).to_bytes()
    assert res[2] == Z.compress(x2).to_bytes()


def test_served_stream_slice_at_real_sizes():
    """The first 60 requests of the served-stream trace (seed 4) at their real
    sizes (log-uniform 64 KiB - 2 GiB, BF16/FP16/FP32, 15% deltas), submitted
    as one burst to a 4-slot server whose budget holds the largest request plus
    1 GiB, so requests queue and batch.  Every compress result must equal the
    direct C-ABI container byte for byte and match the oracle on sampled
    chunks (first, last, one random); every decompress result must equal its
    input."""
    import time
    from tests.test_gpu_parity import _check_sampled_chunks
    torch.cuda.set_device(0)
    trace = W.request_trace(seed=4)[:60]
    inputs = W.serve_inputs(trace, device="cuda")
    containers, need = {}, 0
    a256 = lambda v: (v + 255) // 256 * 256
    for r in trace:
        x, b = inputs(r)
        code = Z.dtype_code(x, None)
        if r.op == "decompress":
            containers[r.rid] = Z.compress(x, base=b)
            need = max(need, containers[r.rid].nbytes + r.nbytes)
        else:
            need = max(need, r.nbytes + a256(Z.compress_bound(r.nbytes, code, Z.DEFAULT_CHUNK))
                       + a256(Z.workspace_size(r.nbytes, code, Z.DEFAULT_CHUNK)))
    assert max(r.nbytes for r in trace) > (1 << 30)       # the slice reaches GiB sizes
    s = Z.Server(need + (1 << 30), slots=4)
    for r in trace:
        x, b = inputs(r)
        if r.op == "compress":
            s.submit_compress(x, base=b, tag=r.rid)
        else:
            s.submit_decompress(containers[r.rid], base=b, tag=r.rid)
    rng = np.random.default_rng(4)
    seen, t_end = set(), time.time() + 600
    while len(seen) < len(trace):
        assert time.time() < t_end, "server did not finish"
        for c in s.poll():
            assert c.status == 0, (c.tag, c.status)
            r = trace[c.tag]
            x, b = inputs(r)
            got = s.output(c)
            if r.op == "compress":
                direct = Z.compress(x, base=b)
                assert got.numel() == direct.nbytes
                assert torch.equal(got, direct.device_tensor()), r.rid
                data = x if b is None else (x.view(torch.uint8) ^ b.view(torch.uint8))
                n = direct.zs.n_chunks
                chunks = sorted({0, n - 1, int(rng.integers(0, n))})
                _check_sampled_chunks(direct, data, Z.dtype_code(x, None), chunks)
                del direct
            else:
                assert torch.equal(got, x.contiguous().view(-1).view(torch.uint8)), r.rid
            seen.add(c.tag)
            s.release(c.id)
        time.sleep(0.001)
    st = s.stats()
    s.close()
    assert st.completed == len(trace) and st.max_batch > 1
