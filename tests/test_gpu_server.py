"""The sort server (ps_server_*): requests of mixed sizes, dtypes and pivot
modes, submitted from several threads while earlier ones are on the GPU, must
each come out exactly as the oracle sorts them (the unique ascending
permutation, Sec. 2) and exactly as ps_sort sorts them alone on the GPU (the
same result alone and in the mix); admission respects the memory budget;
close drains everything admitted and queued."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

DT = ["int32", "int64", "float32", "float64"]
DISTS = ["uniform", "sorted", "reverse", "few_unique"]


@pytest.fixture(scope="module")
def ps():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2305_05245_gb300 as ps
    assert torch.cuda.is_available()
    return ps


def make_requests(n_req, seed, max_log=20):
    import torch
    z = synth.splitmix64(seed, 3 * n_req)
    reqs = []
    for i in range(n_req):
        u = float(z[3 * i] >> np.uint64(11)) * 2.0 ** -53
        n = int(2.0 ** (max_log * u)) - 1
        dt = DT[int(z[3 * i + 1] % np.uint64(4))]
        dist = DISTS[int(z[3 * i + 2] % np.uint64(4))]
        mode = "exact" if i % 3 else "regular"
        x = synth.keys_torch(n, dt, dist, seed=synth.seed_for("srv", seed, i)) if n else \
            torch.empty(0, dtype=getattr(torch, dt), device="cuda")
        reqs.append((x, mode))
    torch.cuda.synchronize()
    return reqs


def alone(ps, reqs):
    import torch
    out = []
    for x, mode in reqs:
        y = x.clone()
        if y.numel() > 1:
            ps.sort(y, mode)
        out.append(y)
    torch.cuda.synchronize()
    return out


DT_CODE = {"int32": 0, "int64": 1, "float32": 2, "float64": 3}


def oracle_results(ora, reqs):
    """Each request's expected output from the oracle, computed on a host copy
    of its input: the plain definition for every request, and for the small
    ones also the four-step oracle run with the (n_B, n_P) the library
    resolves for that size."""
    import paper_2305_05245_gb300 as ps
    out = []
    for x, mode in reqs:
        host = x.cpu().numpy()
        want = ora.reference_sort(host)
        if 1 < host.size <= (1 << 14):
            nb, npart = ps.resolve_params(host.size, DT_CODE[str(host.dtype)])
            r = ora.sort(host, 1 if mode == "exact" else 0, nb, npart)
            assert r.out.tobytes() == want.tobytes()
        out.append(want)
    return out


def assert_oracle(work, oracle_want):
    for i, (w, y) in enumerate(zip(work, oracle_want)):
        assert w.cpu().numpy().tobytes() == y.tobytes(), "request %d differs from the oracle" % i


def wait_all(srv, ids, timeout=120.0):
    got = {}
    t0 = time.time()
    while len(got) < len(ids):
        for rid, st in srv.poll():
            got[rid] = st
        if time.time() - t0 > timeout:
            raise AssertionError("server did not finish %d requests in %.0f s" % (len(ids) - len(got), timeout))
        time.sleep(0.001)
    return got


def test_server_mixed_requests_equal_alone(ps, ora):
    import torch
    reqs = make_requests(300, 1)
    owant = oracle_results(ora, reqs)
    want = alone(ps, reqs)
    work = [x.clone() for x, _ in reqs]
    torch.cuda.synchronize()
    srv = ps.Server(budget_bytes=8 << 30, max_inflight=64)
    try:
        ids = [srv.submit(w, mode) for w, (_, mode) in zip(work, reqs)]
        got = wait_all(srv, ids)
    finally:
        srv.close()
    assert all(got[i] == 0 for i in ids)
    assert_oracle(work, owant)
    for w, y in zip(work, want):
        assert torch.equal(w, y)


def test_server_concurrent_submitters(ps, ora):
    import torch
    reqs = make_requests(200, 2, max_log=18)
    owant = oracle_results(ora, reqs)
    want = alone(ps, reqs)
    work = [x.clone() for x, _ in reqs]
    torch.cuda.synchronize()
    srv = ps.Server(budget_bytes=2 << 30, max_inflight=16)
    ids = [None] * len(reqs)

    def submitter(k):
        for i in range(k, len(reqs), 4):
            ids[i] = srv.submit(work[i], reqs[i][1])

    th = [threading.Thread(target=submitter, args=(k,)) for k in range(4)]
    try:
        for t in th:
            t.start()
        for t in th:
            t.join()
        got = wait_all(srv, ids)
    finally:
        srv.close()
    assert sorted(got) == sorted(ids) and all(st == 0 for st in got.values())
    assert_oracle(work, owant)
    for w, y in zip(work, want):
        assert torch.equal(w, y)


def test_server_budget_and_close_drains(ps, ora):
    import torch
    from paper_2305_05245_gb300 import PsortError
    srv = ps.Server(budget_bytes=64 << 20, max_inflight=4)
    big = torch.zeros(1 << 24, dtype=torch.int64, device="cuda")  # 128 MiB of keys > budget
    with pytest.raises(PsortError):
        srv.submit(big, "exact")
    reqs = make_requests(40, 3, max_log=16)
    owant = oracle_results(ora, reqs)
    want = alone(ps, reqs)
    work = [x.clone() for x, _ in reqs]
    torch.cuda.synchronize()
    for w, (_, mode) in zip(work, reqs):
        srv.submit(w, mode)
    srv.close()  # waits for every queued and admitted request
    torch.cuda.synchronize()
    assert_oracle(work, owant)
    for w, y in zip(work, want):
        assert torch.equal(w, y)


def test_server_failed_round_does_not_stop_the_others(ps, ora):
    """A round that fails at launch (injected on the host) completes its
    requests with an error status, leaves their keys untouched, and the
    server goes on serving correctly."""
    import torch
    reqs = make_requests(40, 5, max_log=18)
    owant = oracle_results(ora, reqs)
    want = alone(ps, reqs)
    work = [x.clone() for x, _ in reqs]
    torch.cuda.synchronize()
    srv = ps.Server(budget_bytes=8 << 30, max_inflight=1)  # one request per round
    try:
        srv.debug_fail("rounds", 3)
        ids = [srv.submit(w, mode) for w, (_, mode) in zip(work, reqs)]
        got = wait_all(srv, ids)
    finally:
        srv.close()
    torch.cuda.synchronize()
    failed = [i for i, rid in enumerate(ids) if got[rid] != 0]
    # the first three admitted rounds (one request of more than one key each) fail
    multi = [i for i, (x, _) in enumerate(reqs) if x.numel() > 1]
    assert failed == multi[:3]
    for i, (w, (x, _)) in enumerate(zip(work, reqs)):
        if i in failed:
            assert torch.equal(w, x), "a failed request's keys changed"
        else:
            assert got[ids[i]] == 0 and torch.equal(w, want[i])
            assert w.cpu().numpy().tobytes() == owant[i].tobytes()


def test_server_survives_failed_streams(ps, ora):
    """Two of the three stream slots retired (injected): results stay exact on
    the last one.  All three retired: queued and new requests fail with
    PS_ERR_CUDA and close still returns."""
    import torch
    reqs = make_requests(30, 9, max_log=18)
    owant = oracle_results(ora, reqs)
    want = alone(ps, reqs)
    work = [x.clone() for x, _ in reqs]
    torch.cuda.synchronize()
    srv = ps.Server(budget_bytes=8 << 30, max_inflight=8)
    try:
        srv.debug_fail("streams", 2)
        ids = [srv.submit(w, mode) for w, (_, mode) in zip(work, reqs)]
        got = wait_all(srv, ids)
        assert all(got[r] == 0 for r in ids)
        assert_oracle(work, owant)
        for w, y in zip(work, want):
            assert torch.equal(w, y)
        srv.debug_fail("streams", 1)
        time.sleep(0.2)
        x = synth.keys_torch(100_000, "int64", "uniform", seed=3)
        before = x.clone()
        rid = srv.submit(x, "exact")
        got = wait_all(srv, [rid])
        assert got[rid] == -4  # PS_ERR_CUDA
        torch.cuda.synchronize()
        assert torch.equal(x, before)
    finally:
        srv.close()
