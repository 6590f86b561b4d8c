"""The request server (psht_server_*) through the C ABI (marked gpu): results of requests run in a
concurrent mix equal those run alone, the plan cache and the memory admission (eviction, a request
that can never fit), and the error path of an invalid request."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fields(n_fields=5, seed=3):
    from paper_2603_17166_gb300 import synthetic as S

    gen = np.random.default_rng(seed)
    out = []
    for i in range(n_fields):
        lmax = int(gen.choice([48, 96, 160]))
        s = int(gen.choice([0, 2]))
        eps = float(gen.choice([1e-5, 1e-10]))
        n = int(gen.integers(2000, 20000))
        th, ph = S.patch_points(n, "cap" if i % 2 else "box", float(gen.uniform(-90, -30)),
                                float(gen.uniform(0.002, 0.04)), gen)
        cd = torch.complex64 if eps >= 1e-5 else torch.complex128
        na = S.nalm(lmax)
        out.append(dict(key=100 + i, lmax=lmax, s=s, eps=eps, cd=cd,
                        theta=torch.from_numpy(th).cuda(), phi=torch.from_numpy(ph).cuda(),
                        g=torch.from_numpy(S.gaussian_alm(lmax, s, gen, "white")).cuda().to(cd),
                        c=torch.from_numpy(S.gaussian_alm(lmax, s, gen, "white")).cuda().to(cd) if s else None,
                        f=torch.from_numpy(gen.standard_normal(n) + 1j * gen.standard_normal(n)).cuda().to(cd),
                        na=na, n=n))
    return out


def _submit(srv, fd, op):
    from paper_2603_17166_gb300 import Server

    if op == 0:
        out = torch.empty(fd["n"], dtype=fd["cd"], device="cuda")
        t = srv.submit(Server.SYNTHESIS, fd["key"], fd["s"], fd["lmax"], fd["eps"], fd["theta"], fd["phi"],
                       fd["g"], fd["c"], out)
        return t, (out,)
    go = torch.empty(fd["na"], dtype=fd["cd"], device="cuda")
    co = torch.empty(fd["na"], dtype=fd["cd"], device="cuda") if fd["s"] else None
    t = srv.submit(Server.ADJOINT, fd["key"], fd["s"], fd["lmax"], fd["eps"], fd["theta"], fd["phi"], fd["f"],
                   None, go, co)
    return t, (go, co)


def _close(a, b, fd):
    tol = 1e-12 if fd["cd"] == torch.complex128 else 1e-5
    for x, y in zip(a, b):
        if x is None:
            continue
        num = torch.linalg.vector_norm((x - y).to(torch.complex128))
        den = torch.linalg.vector_norm(y.to(torch.complex128))
        assert float(num) <= tol * float(den), (fd["key"], float(num / den))


def test_mix_matches_alone():
    """20 requests replayed alone (one worker) and then all at once on four workers."""
    from paper_2603_17166_gb300 import Server

    fields = _fields()
    gen = np.random.default_rng(9)
    reqs = [(int(gen.integers(len(fields))), int(gen.integers(2))) for _ in range(20)]
    srv1 = Server(nstreams=1)
    alone = []
    for i, op in reqs:
        t, out = _submit(srv1, fields[i], op)
        r = srv1.wait(t)
        assert r["status"] == 0
        alone.append(out)
    srv1.close()
    srv4 = Server(nstreams=4)
    pend = [_submit(srv4, fields[i], op) for i, op in reqs]
    res = [(srv4.wait(t), out) for t, out in pend]
    st = srv4.stats()
    srv4.close()
    for (i, op), (r, out), ref in zip(reqs, res, alone):
        assert r["status"] == 0
        if op == 0:  # synthesis has a fixed summation order: identical bits
            assert torch.equal(out[0], ref[0])
        else:        # the adjoint's spreading uses atomics: equal up to the summation order
            _close(out, ref, fields[i])
    assert st["completed"] == 20 and st["failed"] == 0
    assert st["plans_created"] == len({i for i, _ in reqs})
    # every plan call either built its plan or found it cached; a batch of k requests is one call
    assert st["batches"] == st["plans_created"] + st["cache_hits"]
    assert sum(1.0 / r["batch"] for r, _ in res) == pytest.approx(st["batches"])
    assert len({r["worker"] for r, _ in res}) > 1


def test_budget_evicts_and_rejects():
    from paper_2603_17166_gb300 import Server, estimate_points

    fields = _fields(4, seed=4)
    sizes = [estimate_points(fd["s"], fd["lmax"], fd["theta"], fd["phi"], fd["eps"]) for fd in fields]
    budget = max(sizes) + min(sizes) // 2  # room for one plan at a time (plus slack)
    srv = Server(nstreams=2, budget_bytes=budget)
    outs = []
    for rep in range(2):
        for fd in fields:
            t, out = _submit(srv, fd, 0)
            r = srv.wait(t)
            assert r["status"] == 0
            outs.append(out[0].clone())
    st = srv.stats()
    assert st["evictions"] >= len(fields)
    assert st["bytes_peak"] <= budget
    for k in range(len(fields)):  # a plan rebuilt after eviction gives the same result
        assert torch.equal(outs[k], outs[k + len(fields)])
    srv.close()
    tiny = Server(nstreams=1, budget_bytes=1024)
    t, _ = _submit(tiny, fields[0], 0)
    r = tiny.wait(t)
    assert r["status"] == -12  # PSHT_ENOMEM: can never fit
    tiny.close()


def test_invalid_request_fails_alone():
    from paper_2603_17166_gb300 import Server

    fd = _fields(1, seed=5)[0]
    bad = dict(fd)
    bad["key"] = 999
    bad["theta"] = fd["theta"].clone()
    bad["theta"][0] = float("nan")
    srv = Server(nstreams=2)
    t_bad, _ = _submit(srv, bad, 0)
    t_ok, _ = _submit(srv, fd, 0)
    assert srv.wait(t_bad)["status"] == -22  # PSHT_EINVAL from the point validation
    assert srv.wait(t_ok)["status"] == 0
    srv.close()


def test_reused_key_with_other_point_count_gets_its_own_plan():
    """A points_key reused for a smaller point set must not run the plan cached for the larger one
    (that plan writes its own npts values): the point count is part of the cache key, so the
    second request builds a plan of its own and its result equals that request run alone."""
    from paper_2603_17166_gb300 import Server

    fd = _fields(1, seed=6)[0]
    small = dict(fd)
    k = fd["n"] // 3
    small.update(theta=fd["theta"][:k].clone(), phi=fd["phi"][:k].clone(), f=fd["f"][:k].clone(), n=k)
    srv = Server(nstreams=1)
    t, out_big = _submit(srv, fd, 0)
    assert srv.wait(t)["status"] == 0
    t, out_small = _submit(srv, small, 0)
    r = srv.wait(t)
    assert r["status"] == 0 and r["plan_cached"] == 0
    assert out_small[0].numel() == k
    t, adj_small = _submit(srv, small, 1)
    assert srv.wait(t)["status"] == 0
    assert srv.stats()["plans_created"] == 2
    srv.close()
    ref = Server(nstreams=1)
    t, out_ref = _submit(ref, small, 0)
    assert ref.wait(t)["status"] == 0
    t, adj_ref = _submit(ref, small, 1)
    assert ref.wait(t)["status"] == 0
    ref.close()
    assert torch.equal(out_small[0], out_ref[0])
    _close(adj_small, adj_ref, small)
    # the larger set's own result is the head of nothing in particular: only check it is finite
    assert torch.isfinite(torch.view_as_real(out_big[0])).all()


def test_queued_requests_on_one_plan_run_batched():
    """Requests for one plan and operation that queue up while the plan is busy join the next call as
    a batch (continuous batching); each result equals the same request run alone."""
    from paper_2603_17166_gb300 import Server

    fd = _fields(1, seed=7)[0]
    gen = np.random.default_rng(10)
    gs = [torch.from_numpy(np.ascontiguousarray(
        (gen.standard_normal(fd["na"]) + 1j * gen.standard_normal(fd["na"])))).cuda().to(fd["cd"])
          for _ in range(6)]
    for g in gs:
        g[: fd["lmax"] + 1] = g[: fd["lmax"] + 1].real.to(fd["cd"])
    srv1 = Server(nstreams=1)
    alone = []
    for g in gs:
        f = dict(fd)
        f["g"] = g
        t, out = _submit(srv1, f, 0)
        assert srv1.wait(t)["status"] == 0
        alone.append(out[0])
    srv1.close()
    srv = Server(nstreams=1)
    pend = []
    for g in gs:  # submitted back to back: the first runs, the others queue behind it
        f = dict(fd)
        f["g"] = g
        pend.append(_submit(srv, f, 0))
    res = [(srv.wait(t), out) for t, out in pend]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r, _ in res)
    assert max(r["batch"] for r, _ in res) > 1
    assert st["batched_requests"] >= 2 and st["batches"] < len(gs)
    for (r, out), ref in zip(res, alone):
        assert torch.equal(out[0], ref)


def test_batch_limit_one_runs_every_request_alone():
    """psht_server_set_batch_limit(1): queued requests for one plan still run, one call each; the limit
    is checked (1..8)."""
    from paper_2603_17166_gb300 import PshtError, Server

    fd = _fields(1, seed=8)[0]
    srv = Server(nstreams=1, max_batch=1)
    pend = [_submit(srv, fd, 0) for _ in range(4)]
    res = [(srv.wait(t), out) for t, out in pend]
    st = srv.stats()
    assert all(r["status"] == 0 and r["batch"] == 1 for r, _ in res)
    assert st["batched_requests"] == 0 and st["batches"] == 4
    for r, out in res[1:]:
        assert torch.equal(out[0], res[0][1][0])
    for bad in (0, 9):
        with pytest.raises(PshtError):
            srv.set_batch_limit(bad)
    srv.close()
