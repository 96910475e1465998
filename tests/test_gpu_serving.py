"""GPU tests of the retrieval server (request loop with plane caches).

Every request's result must be the same alone and in a concurrent mix: the
mix runs on several worker streams with caches kept and evicted under a small
HBM budget, the reference runs each request alone on the plain per-request
path.  Field requests are also checked against the oracle bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2505_00227_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def setup(B):
    from paper_2505_00227_gb300 import synthetic as S
    ctx = B.Context()
    fields = {
        "a": S.spectral((24, 32, 64), seed=41).numpy(),
        "b": S.blobs((17, 23, 30), seed=42).numpy(),
        "c": S.spectral((16, 16, 128), seed=43).numpy(),
    }
    vel = S.velocity_triplet((20, 24, 64), seed=44)
    vel = [v.numpy() for v in vel]
    hs = {k: ctx.refactor(torch.from_numpy(v).cuda()) for k, v in fields.items()}
    vh = [ctx.refactor(torch.from_numpy(v).cuda()) for v in vel]
    ctx.prepare_vmag(vh, *[torch.from_numpy(v).cuda() for v in vel])
    oracles = {k: O.Field(v) for k, v in fields.items()}
    return ctx, fields, hs, vel, vh, oracles


def _requests(seed, n=40):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        tau = float(10.0 ** rng.uniform(-6, -1))
        if rng.random() < 0.25:
            out.append(("vmag", tau))
        else:
            out.append((str(rng.choice(["a", "b", "c"])), tau))
    return out


def _serve(B, ctx, setup, reqs, budget, slots, keep):
    _, fields, hs, vel, vh, _ = setup
    srv = B.Server(ctx, budget, max_slots=slots, keep_cache=keep)
    for h in list(hs.values()) + vh:
        srv.add(h)
    tickets, outs = [], []
    for name, tau in reqs:
        if name == "vmag":
            o = torch.empty(vel[0].shape, dtype=torch.float32, device="cuda")
            comps = [torch.empty_like(o) for _ in range(3)]
            tickets.append(srv.submit(vh, tau, out=comps, out_vmag=o))
            outs.append((o, comps))
        else:
            o = torch.empty(fields[name].shape, dtype=torch.float32, device="cuda")
            tickets.append(srv.submit([hs[name]], tau, out=o))
            outs.append((o, None))
    res = [srv.poll(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    got = []
    for (o, comps), r in zip(outs, res):
        got.append((o.cpu().numpy(), None if comps is None else [c.cpu().numpy() for c in comps], r))
    return got, stats


def _resident(setup):
    _, _, hs, _, vh, _ = setup
    tot, caches = 0, []
    for h in list(hs.values()) + vh:
        h.compact()
        r, c, m = h.memory()
        tot += r
        caches.append(m)
    return tot, caches


def test_alone_equals_mix(B, setup):
    ctx, fields, hs, vel, vh, oracles = setup
    reqs = _requests(7)
    resident, caches = _resident(setup)
    alone, st1 = _serve(B, ctx, setup, reqs, 1 << 40, 1, False)
    # budget: every stored field + the three largest caches, so the mix evicts
    budget = resident + sum(sorted(caches)[-3:]) + 3 * 4 * vel[0].size
    mix, st2 = _serve(B, ctx, setup, reqs, budget, 4, True)
    assert st1["completed"] == st2["completed"] == len(reqs)
    assert st2["peak"] <= budget
    assert st2["evictions"] > 0
    for (name, tau), (a, ac, ra), (m, mc, rm) in zip(reqs, alone, mix):
        assert ra[0] == rm[0]
        assert np.array_equal(a.view(np.uint32), m.view(np.uint32)), (name, tau)
        if ac is not None:
            for x, y in zip(ac, mc):
                assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
            assert ra[1][3].est_linf == rm[1][3].est_linf
        else:
            F = oracles[name]
            rc, ref, g, E = F.retrieve(tau * F.range)
            assert rm[0] == rc and rm[1][0].groups == list(g) and rm[1][0].est_linf == E
            assert np.array_equal(m.view(np.uint32), ref.view(np.uint32))
            err = np.abs(m.astype(np.float64) - fields[name].astype(np.float64)).max()
            assert err <= rm[1][0].est_linf
        t_submit, t_start, t_done = rm[2]
        assert t_submit <= t_start <= t_done


def test_cache_saves_decoding(B, setup):
    ctx, fields, hs, vel, vh, oracles = setup
    srv = B.Server(ctx, 1 << 40, max_slots=2, keep_cache=True)
    h = hs["a"]
    srv.add(h)
    h.drop_cache()
    o = torch.empty(fields["a"].shape, dtype=torch.float32, device="cuda")
    st, inf1, _ = srv.poll(srv.submit([h], 1e-3, out=o))
    st, inf2, _ = srv.poll(srv.submit([h], 1e-3, out=o))
    assert inf1[0].bytes_fetched_new > 0 and inf2[0].bytes_fetched_new == 0
    st, inf3, _ = srv.poll(srv.submit([h], 1e-5, out=o))
    assert 0 < inf3[0].bytes_fetched_new < inf3[0].bytes_fetched_total
    srv.close()


def test_admission_errors(B, setup):
    ctx, fields, hs, vel, vh, _ = setup
    srv = B.Server(ctx, 1024, max_slots=1)
    with pytest.raises(B.HpmdrError) as e:
        srv.add(hs["b"])
    assert e.value.status == B.ERR_NOMEM
    srv.close()
    srv = B.Server(ctx, 1 << 40, max_slots=1)
    o = torch.empty(fields["b"].shape, dtype=torch.float32, device="cuda")
    with pytest.raises(B.HpmdrError) as e:
        srv.submit([hs["b"]], 1e-3, out=o)  # never added
    assert e.value.status == B.ERR_ARG
    srv.close()


def test_cancel_queued_requests(B, setup):
    """Host-side cancellation: a request still queued is dropped and polls as
    cancelled; one that already started completes with its normal result."""
    ctx, fields, hs, vel, vh, oracles = setup
    srv = B.Server(ctx, 1 << 40, max_slots=1, keep_cache=False)
    srv.add(hs["a"])
    F = oracles["a"]
    rc, ref, g, E = F.retrieve(1e-6 * F.range)
    outs = [torch.empty(fields["a"].shape, dtype=torch.float32, device="cuda") for _ in range(24)]
    tickets = [srv.submit([hs["a"]], 1e-6, out=o) for o in outs]  # one slot, one handle: serial
    cancelled = [srv.cancel(t) for t in tickets[8:]]
    assert any(cancelled)  # the last of 24 serial requests cannot all have started
    for i, (t, o) in enumerate(zip(tickets, outs)):
        st, info, times = srv.poll(t)
        if i >= 8 and cancelled[i - 8]:
            assert st == B.ERR_CANCELLED
        else:
            assert st == rc == 0 and info[0].groups == list(g)
            assert np.array_equal(o.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    with pytest.raises(B.HpmdrError) as e:
        srv.cancel(tickets[0])  # already polled
    assert e.value.status == B.ERR_ARG
    assert srv.stats()["queued"] == 0
    srv.close()


def test_queue_deadline_times_out_waiting_requests(B, setup):
    """A request still queued past the server's deadline fails with
    ERR_TIMEOUT instead of starting; requests that ran are exact."""
    ctx, fields, hs, vel, vh, oracles = setup
    srv = B.Server(ctx, 1 << 40, max_slots=1, keep_cache=False, queue_timeout_s=1e-3)
    srv.add(hs["c"])
    F = oracles["c"]
    rc, ref, g, E = F.retrieve(1e-5 * F.range)
    outs = [torch.empty(fields["c"].shape, dtype=torch.float32, device="cuda") for _ in range(64)]
    tickets = [srv.submit([hs["c"]], 1e-5, out=o) for o in outs]
    res = [srv.poll(t) for t in tickets]
    assert {r[0] for r in res} <= {0, B.ERR_TIMEOUT}
    assert any(r[0] == B.ERR_TIMEOUT for r in res) and any(r[0] == 0 for r in res)
    for (st, info, times), o in zip(res, outs):
        if st == 0:
            assert info[0].groups == list(g)
            assert np.array_equal(o.cpu().numpy().view(np.uint32), ref.view(np.uint32))
        else:
            assert times[2] - times[0] >= 1e-3  # failed only after its deadline
    srv.close()
    with pytest.raises(B.HpmdrError):
        B.Server(ctx, 1 << 40, queue_timeout_s=-1.0)
