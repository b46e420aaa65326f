"""The serving engine (mm_serve_submit / mm_serve_poll): results within each
class's bound, the same alone and in a mix, admission under a memory budget,
ticket semantics, concurrent submitters, and destroy with queued work."""
import threading
import time

import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

from gpu_util import bound_ok

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODE = {0: "fp64", 1: "fp64_emu", 2: "fp32_emu"}


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_15384_gb300 as mm
    from paper_2408_15384_gb300 import build
    build.build()
    return mm


def make_requests(count, lo, hi, seed):
    dims = inputs.problem_set(count, lo, hi, seed)
    classes = (inputs.unit(seed, inputs.STREAM_CLASS, count) < 0.5).astype(int)  # 1 = FP64-accuracy, 0 = FP32
    reqs = []
    for i, (m, n, k) in enumerate(dims):
        A = inputs.uniform(int(m), int(k), seed * 7919 + i, inputs.STREAM_A)
        B = inputs.uniform(int(k), int(n), seed * 7919 + i, inputs.STREAM_B)
        prec = 1 if classes[i] else 2
        if i % 11 == 5:
            prec = 0
        reqs.append((A, B, prec))
    return reqs


def wait_all(h, tickets, timeout=120.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t in done:
                continue
            rc, st = h.serve_poll(t)
            if rc != 1:
                done[t] = (rc, st)
        time.sleep(0.001)
    return done


def test_serve_mixed_results_and_alone_vs_mix(mm):
    reqs = make_requests(60, 16, 400, 3)
    with mm.Handle(0) as h:
        dev = []
        tickets = []
        for i, (A, B, prec) in enumerate(reqs):
            Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            Cd = torch.full((A.shape[0], B.shape[1]), np.nan, dtype=torch.float64, device="cuda")
            dev.append((Ad, Bd, Cd))
        torch.cuda.synchronize()
        for i, ((Ad, Bd, Cd), (_, _, prec)) in enumerate(zip(dev, reqs)):
            tickets.append(h.serve_submit(Ad, Bd, Cd, precision=prec, tag=1000 + i))
        done = wait_all(h, tickets)
        assert len(done) == len(tickets)
        for i, t in enumerate(tickets):
            rc, st = done[t]
            assert rc == 0 and st.user_tag == 1000 + i
            assert st.t_submit_us <= st.t_admit_us <= st.t_launch_us <= st.t_done_us
        mixed = [Cd.cpu().numpy() for (_, _, Cd) in dev]
        for (A, B, prec), C in zip(reqs, mixed):
            assert bound_ok(C, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(A.shape[1], MODE[prec]))
        # the same requests served alone give the same bits
        for i in range(0, len(reqs), 6):
            Ad, Bd, _ = dev[i]
            Ca = torch.full_like(dev[i][2], np.nan)
            t = h.serve_submit(Ad, Bd, Ca, precision=reqs[i][2])
            h.serve_drain()
            rc, _ = h.serve_poll(t)
            assert rc == 0
            assert np.array_equal(Ca.cpu().numpy(), mixed[i])


def test_serve_budget_admission(mm):
    # a 48 MiB budget: requests of ~7 MiB each must wait for earlier ones to finish
    with mm.Handle(0, budget_bytes=48 << 20) as h:
        m = n = k = 384
        A = inputs.uniform(m, k, 1, inputs.STREAM_A)
        B = inputs.uniform(k, n, 1, inputs.STREAM_B)
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        Cs = [torch.empty((m, n), dtype=torch.float64, device="cuda") for _ in range(16)]
        tickets = [h.serve_submit(Ad, Bd, C, precision=1) for C in Cs]
        done = wait_all(h, tickets)
        assert all(done[t][0] == 0 for t in tickets)
        ref = oracle.gemm(A, B)
        D = oracle.absprod(A, B)
        for C in Cs:
            assert bound_ok(C.cpu().numpy(), ref, D, em.gamma(k, "fp64_emu"))
        big = torch.empty((4096, 4096), dtype=torch.float64, device="cuda")
        big2 = torch.empty((4096, 4096), dtype=torch.float64, device="cuda")
        big3 = torch.empty((4096, 4096), dtype=torch.float64, device="cuda")
        with pytest.raises(mm.MMError) as ei:
            h.serve_submit(big, big2, big3, precision=1)
        assert ei.value.status == 3


def test_serve_tickets_and_threads(mm):
    with mm.Handle(0) as h:
        assert h.serve_poll(12345)[0] == 7          # unknown ticket
        A = torch.from_numpy(inputs.uniform(64, 80, 2, inputs.STREAM_A)).cuda()
        B = torch.from_numpy(inputs.uniform(80, 72, 2, inputs.STREAM_B)).cuda()
        outs, tickets, lock = [], [], threading.Lock()

        def worker(seed):
            for j in range(20):
                C = torch.empty((64, 72), dtype=torch.float64, device="cuda")
                t = h.serve_submit(A, B, C, precision=(seed + j) % 3)
                with lock:
                    outs.append((t, C, (seed + j) % 3))
                    tickets.append(t)

        ths = [threading.Thread(target=worker, args=(s,)) for s in range(3)]
        [t.start() for t in ths]
        [t.join() for t in ths]
        h.serve_drain()
        assert len(set(tickets)) == 60
        ref, D = oracle.gemm(A.cpu().numpy(), B.cpu().numpy()), oracle.absprod(A.cpu().numpy(), B.cpu().numpy())
        for t, C, prec in outs:
            rc, st = h.serve_poll(t)
            assert rc == 0
            assert h.serve_poll(t)[0] == 7          # released after the first successful poll
            assert bound_ok(C.cpu().numpy(), ref, D, em.gamma(80, MODE[prec]))


def test_destroy_with_queued_requests(mm):
    h = mm.Handle(0)
    A = torch.from_numpy(inputs.uniform(512, 512, 3, inputs.STREAM_A)).cuda()
    B = torch.from_numpy(inputs.uniform(512, 512, 3, inputs.STREAM_B)).cuda()
    Cs = [torch.empty((512, 512), dtype=torch.float64, device="cuda") for _ in range(40)]
    for C in Cs:
        h.serve_submit(A, B, C, precision=1)
    t0 = time.time()
    h.close()                                     # cancels what is queued, finishes what runs
    assert time.time() - t0 < 30


def test_serve_reports_nonfinite_per_request(mm):
    """A served FP64-accuracy request with a NaN entry among clean ones: that
    request polls MM_ERR_NONFINITE, the others MM_OK with their correct
    results, and no error is left behind for any stream of the handle."""
    with mm.Handle(0) as h:
        reqs = []
        for i in range(12):
            A = inputs.uniform(96 + 8 * i, 200, 300 + i, inputs.STREAM_A)
            B = inputs.uniform(200, 80, 300 + i, inputs.STREAM_B)
            if i == 5:
                A[7, 13] = np.nan
            reqs.append((A, B, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                         torch.full((A.shape[0], 80), np.nan, dtype=torch.float64, device="cuda")))
        torch.cuda.synchronize()
        tickets = [h.serve_submit(Ad, Bd, Cd, precision=1) for _, _, Ad, Bd, Cd in reqs]
        done = wait_all(h, tickets)
        assert len(done) == len(tickets)
        for i, t in enumerate(tickets):
            rc, _ = done[t]
            assert rc == (4 if i == 5 else 0), (i, rc)
        for i, (A, B, _, _, Cd) in enumerate(reqs):
            C = Cd.cpu().numpy()
            if i == 5:
                assert np.all(np.isnan(C[7]))
            else:
                assert bound_ok(C, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(200, "fp64_emu"))
        assert h.sync() == 0
        s2 = torch.cuda.Stream()
        assert h.sync(s2) == 0


def test_serve_batches_overlap_while_others_run(mm):
    """Continuous batching: a large FP64-accuracy request goes first; small
    FP32-accuracy requests submitted right after it are admitted and launched
    on other streams while it is still on the GPU, and their device intervals
    overlap its interval. Results stay the same as alone."""
    with mm.Handle(0) as h:
        N = 4096
        Ab = torch.empty((2 * N, N), dtype=torch.float64, device="cuda")
        Bb = torch.empty((N, N), dtype=torch.float64, device="cuda")
        mm.fill_uniform(Ab, 77, inputs.STREAM_A)
        mm.fill_uniform(Bb, 77, inputs.STREAM_B)
        Cb = torch.empty((2 * N, N), dtype=torch.float64, device="cuda")
        small = []
        for i in range(24):
            A = torch.from_numpy(inputs.uniform(128, 256, 900 + i, inputs.STREAM_A)).cuda()
            B = torch.from_numpy(inputs.uniform(256, 192, 900 + i, inputs.STREAM_B)).cuda()
            small.append((A, B, torch.empty((128, 192), dtype=torch.float64, device="cuda")))
        torch.cuda.synchronize()
        tb = h.serve_submit(Ab, Bb, Cb, precision=1)
        ts = []
        for A, B, C in small:
            ts.append(h.serve_submit(A, B, C, precision=2))
            time.sleep(0.0002)
        done = wait_all(h, [tb] + ts)
        rcb, stb = done[tb]
        assert rcb == 0
        later = [done[t][1] for t in ts]
        assert all(done[t][0] == 0 for t in ts)
        # launched while the large batch was in flight, on another stream ...
        during = [st for st in later if st.t_launch_us < stb.t_done_us and st.stream != stb.stream]
        assert during, [(st.t_launch_us, st.stream) for st in later[:4]] + [(stb.t_launch_us, stb.t_done_us, stb.stream)]
        # ... and running on the device inside the large batch's device interval
        assert any(stb.t_gpu_start_us < st.t_gpu_end_us and st.t_gpu_start_us < stb.t_gpu_end_us for st in during)
        # the mix changed no bits
        for (A, B, C) in small[:4]:
            Ca = torch.empty_like(C)
            t = h.serve_submit(A, B, Ca, precision=2)
            h.serve_drain()
            assert h.serve_poll(t)[0] == 0
            assert torch.equal(Ca, C)
