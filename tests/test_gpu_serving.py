"""Serving loop (stn_server_*): requests arrive while others run, are admitted
against a device-memory budget and run concurrently -- engine 0 in the
persistent scheduler, engine 1 on a pool of worker streams running the
full-grid kernels.  Each result must be the same bits alone and in the mix
(compared with the same engine's solver on that request alone: the batched
solver for engine 0, jacobi_solve_refined_f64 / jacobi_solve_f64 for engine 1)
and meet its tolerance on the CPU oracle's independent double residual."""
import threading
import time

import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

L7 = si.LAPLACE7


def bitwise(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def requests(n, seed=31, lo=6, hi=24):
    sizes = si.log_uniform_sizes(n, lo, hi, seed)
    return [si.normal_interior(int(x), int(y), int(z), 1, seed=seed * 1000 + i) for i, (x, y, z) in enumerate(sizes)]


def alone(lib, rhs, refined, tol, engine=0):
    import torch
    u = torch.zeros(rhs.shape, dtype=torch.float64, device="cuda")
    b = torch.from_numpy(rhs).cuda()
    if engine == 1:
        if refined:
            rc, info = lib.jacobi_solve_refined_f64(b, u, L7, 1, tol, 200000, 1e-2, 50, 40)
        else:
            rc, info = lib.jacobi_solve_f64(b, u, L7, 1, tol, 10 ** 6, 50)
        torch.cuda.synchronize()
        return u.cpu().numpy(), info
    if refined:
        rc, infos = lib.jacobi_solve_batched_refined([u], [b], L7, 1, tol, 200000, 1e-2, 50, 40)
    else:
        rc, infos = lib.jacobi_solve_batched_f64([u], [b], L7, 1, tol, 10 ** 6, 50)
    torch.cuda.synchronize()
    return u.cpu().numpy(), infos[0]


@pytest.fixture(params=[0, 1])
def engine(request):
    return request.param


@pytest.mark.parametrize("refined", [True, False])
def test_serving_results_same_alone_and_in_the_mix(lib, cuda, refined, engine):
    tol = 1e-8
    rhss = requests(16)
    got = {}
    with lib.Server(hbm_budget=1 << 30, tol=tol, refined=refined, check_every=50, max_inflight=8,
                    engine=engine) as srv:
        tickets = []
        for i, b in enumerate(rhss):  # arrivals spread over the run
            tickets.append(srv.submit(b))
            time.sleep(0.002 * (i % 3))
        for i, t in enumerate(tickets):
            res = srv.wait(t, 120.0)
            assert res["rc"] == 0 and res["status"] == 0, res
            assert res["latency_s"] >= res["queue_s"] >= 0
            got[i] = (srv.result(t, rhss[i].shape), res)
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == len(rhss) and st["pending"] == 0 and st["running"] == 0
        assert st["bytes_in_use"] == 0
    for i, b in enumerate(rhss):
        u, res = got[i]
        ref, info = alone(lib, b, refined, tol, engine)
        assert bitwise(u, ref), i
        assert res["iters"] == info["iters"] and res["outer"] == info["outer"]
        assert oracle.residual_norm(u, L7, 1, b) / oracle.interior_norm(b, 1) <= tol


def test_serving_admission_respects_budget(lib, cuda, engine):
    rhss = requests(10, seed=41, lo=20, hi=28)
    per = 3 * 8 * max(b.size for b in rhss) + 3 * 4 * max(b.size for b in rhss) + (1 << 16)
    budget = int(per * 1.5)  # room for the largest request plus a small one
    with lib.Server(hbm_budget=budget, tol=1e-8, refined=True, max_inflight=8, engine=engine) as srv:
        tickets = [srv.submit(b) for b in rhss]
        peak_pending, peak_bytes = 0, 0
        done = 0
        deadline = time.time() + 120
        while done < len(tickets) and time.time() < deadline:
            st = srv.stats()
            peak_pending = max(peak_pending, st["pending"])
            peak_bytes = max(peak_bytes, st["bytes_in_use"])
            done = st["completed"]
            time.sleep(0.001)
        assert done == len(tickets)
        assert peak_bytes <= budget  # never over the budget
        assert peak_pending >= len(tickets) - 3  # requests waited for memory
        for t, b in zip(tickets, rhss):
            res = srv.wait(t, 10.0)
            assert res["status"] == 0
            u = srv.result(t, b.shape)
            assert oracle.residual_norm(u, L7, 1, b) / oracle.interior_norm(b, 1) <= 1e-8


def test_serving_rejects_oversize_and_concurrent_submitters(lib, cuda, engine):
    big = np.zeros(si.padded_shape(64, 64, 64, 1))
    with lib.Server(hbm_budget=1 << 20, tol=1e-6, refined=True, max_inflight=4, engine=engine) as srv:
        with pytest.raises(lib.StencilError) as ei:
            srv.submit(big)
        assert ei.value.code == lib.STN_EBUSY
    # several host threads submitting at once
    rhss = requests(12, seed=51, lo=6, hi=14)
    out = [None] * len(rhss)
    with lib.Server(hbm_budget=1 << 28, tol=1e-8, refined=False, max_inflight=4, engine=engine) as srv:
        def worker(k):
            for i in range(k, len(rhss), 3):
                t = srv.submit(rhss[i])
                out[i] = srv.wait(t, 60.0)
        th = [threading.Thread(target=worker, args=(k,)) for k in range(3)]
        for x in th:
            x.start()
        for x in th:
            x.join()
    assert all(r is not None and r["status"] == 0 for r in out)


def test_serving_shutdown_with_requests_in_flight(lib, cuda, engine):
    rhss = requests(6, seed=61, lo=10, hi=20)
    srv = lib.Server(hbm_budget=1 << 28, tol=1e-8, refined=True, max_inflight=2, engine=engine)
    for b in rhss:
        srv.submit(b)
    t0 = time.time()
    srv.close()  # finishes the submitted requests, then frees everything
    assert time.time() - t0 < 120


def test_serving_survives_injected_admission_failures(lib, cuda, engine):
    """Host-side fault injection: the first admission allocations fail; the
    server retries them later and every request still completes correctly."""
    rhss = requests(6, seed=71, lo=8, hi=16)
    lib.stencil_tune_set("fault_admit_fail", 5)
    before = lib.stencil_tune_get("fault_admit_failed")
    try:
        with lib.Server(hbm_budget=1 << 28, tol=1e-8, refined=True, max_inflight=4, engine=engine) as srv:
            tickets = [srv.submit(b) for b in rhss]
            for t, b in zip(tickets, rhss):
                res = srv.wait(t, 60.0)
                assert res["status"] == 0
                u = srv.result(t, b.shape)
                assert oracle.residual_norm(u, L7, 1, b) / oracle.interior_norm(b, 1) <= 1e-8
    finally:
        lib.stencil_tune_set("fault_admit_fail", 0)
    assert lib.stencil_tune_get("fault_admit_failed") - before == 5


def test_plain_solve_continued_equals_direct(lib, cuda):
    """The bench's plain per-request path solves to 1e-8, copies out, and
    continues from that iterate to 1e-10: groups of check_every sweeps start
    at the same sweeps as in a direct solve to 1e-10, so the continued solve
    ends at the same iterate, bit for bit, after the same number of sweeps."""
    import torch
    for i, b in enumerate(requests(3, seed=81, lo=12, hi=30)):
        d_b = torch.from_numpy(b).cuda()
        u1 = torch.zeros_like(d_b)
        rc1, i1 = lib.jacobi_solve_f64(d_b, u1, L7, 1, 1e-8, 10 ** 7, 50)
        rc2, i2 = lib.jacobi_solve_f64(d_b, u1, L7, 1, 1e-10, 10 ** 7, 50)
        u3 = torch.zeros_like(d_b)
        rc3, i3 = lib.jacobi_solve_f64(d_b, u3, L7, 1, 1e-10, 10 ** 7, 50)
        assert rc1 == rc2 == rc3 == 0
        assert i1["iters"] + i2["iters"] == i3["iters"], (i1, i2, i3)
        assert bitwise(u1.cpu().numpy(), u3.cpu().numpy()), i
