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
