"""Continuous-batching server: results in the mix equal results alone, memory
admission holds, and bad requests fail alone (faults injected on the host)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import laplace, stokes  # noqa: E402
from paper_1507_05925_gb300 import bie  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def requests_():
    rng = np.random.default_rng(41)
    return [synth.random_request(rng, max_bodies=12, nodes=(64, 128)) for _ in range(24)]


def _host(g):
    return {k: np.ascontiguousarray(g[k]) for k in ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")}


def _load(g):
    return np.ascontiguousarray(g["q"] if g["kind"] == 0 else g["FT"].reshape(-1))


def _nout(g):
    n = g["body_start"].size - 1
    return n if g["kind"] == 0 else 3 * n


@pytest.fixture(scope="module")
def alone(requests_):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05925_gb300 import build
    build.build()
    ctx = bie.Context(0)
    outs = []
    for g in requests_:
        out = np.empty(_nout(g))
        fn = bie.elastance_solve if g["kind"] == 0 else bie.mobility_solve
        rc, _ = fn(ctx, _host(g), _load(g), out, opts=bie.make_opts(precision=bie.MIXED_FF))
        assert rc == bie.OK
        outs.append(out)
    ctx.close()
    return outs


def test_results_in_the_mix_equal_results_alone(requests_, alone):
    srv = bie.Server(0, workers=6)
    outs, tickets = [], []
    for i, g in enumerate(requests_):
        out = np.full(_nout(g), np.nan)
        # alternate host and device arrays
        geom = _host(g) if i % 2 == 0 else {k: torch.from_numpy(v).cuda() for k, v in _host(g).items()}
        t = srv.submit(g["kind"], geom, _load(g), out, opts=bie.make_opts(precision=bie.MIXED_FF))
        assert t > 0
        outs.append(out)
        tickets.append(t)
    for t, out, ref in zip(tickets, outs, alone):
        rc, info, sec = srv.wait(t)
        assert rc == bie.OK and sec > 0
        assert np.array_equal(out, ref)  # bitwise: fixed-order reductions
    st = srv.stats()
    assert st["completed"] == len(requests_) and st["inflight_bytes"] == 0
    srv.close()


def test_results_match_the_oracle(requests_, alone):
    for g, out in list(zip(requests_, alone))[:4]:
        if g["kind"] == 0:
            ref = laplace.solve(g, g["q"])["phi"]
        else:
            ref = stokes.solve(g, g["FT"])["UW"].reshape(-1)
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-10


def test_memory_admission_cap(requests_, alone):
    needs = [bie.workspace_bytes(g["kind"], g["body_start"].size - 1, g["x"].size) for g in requests_]
    cap = int(1.5 * max(needs))
    srv = bie.Server(0, workers=8, hbm_cap_bytes=cap)
    outs = [np.empty(_nout(g)) for g in requests_]
    tickets = [srv.submit(g["kind"], _host(g), _load(g), o, opts=bie.make_opts(precision=bie.MIXED_FF))
               for g, o in zip(requests_, outs)]
    for t, out, ref in zip(tickets, outs, alone):
        rc, _, _ = srv.wait(t)
        assert rc == bie.OK
        assert np.array_equal(out, ref)
    st = srv.stats()
    assert st["peak_inflight_bytes"] <= cap
    srv.close()


def test_bad_requests_fail_alone(requests_, alone):
    srv = bie.Server(0, workers=3, hbm_cap_bytes=64 << 20)
    good = requests_[:6]
    bad = dict(_host(requests_[0]))
    bs = bad["body_start"].copy()
    if bs.size > 2:
        bs[1] = 3  # first body has 3 nodes: invalid
    else:
        bs = np.array([0, 3, bs[-1]], dtype=np.int32)
    bad["body_start"] = bs
    huge = synth.assemble([synth.disc(3.0 * i, 0.0, 1.0, 16384) for i in range(16)])  # over 64 MB
    outs = [np.empty(_nout(g)) for g in good]
    tickets = []
    for i, (g, o) in enumerate(zip(good, outs)):
        tickets.append(srv.submit(g["kind"], _host(g), _load(g), o, opts=bie.make_opts(precision=bie.MIXED_FF)))
        if i == 2:
            tb = srv.submit(0, bad, np.zeros(bs.size - 1), np.empty(bs.size - 1))
            assert tb > 0
    assert srv.submit(0, _host(huge), np.zeros(16), np.empty(16)) == bie.ERR_NOMEM
    for t, out, ref in zip(tickets, outs, alone[:6]):
        rc, _, _ = srv.wait(t)
        assert rc == bie.OK and np.array_equal(out, ref)
    assert srv.wait(tb)[0] == bie.ERR_INVALID
    assert srv.wait(tb)[0] == bie.ERR_INVALID  # a ticket can be waited for once
    srv.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("cap_factor", [0, 3])
def test_batching_matches_results_alone(requests_, alone, cap_factor):
    # queued requests of one kind and options are solved together: the results
    # agree with the solo ones to the solve tolerance, memory admission holds
    needs = [bie.workspace_bytes(g["kind"], g["body_start"].size - 1, g["x"].size) for g in requests_]
    cap = int(cap_factor * max(needs))
    srv = bie.Server(0, workers=2, hbm_cap_bytes=cap)
    assert srv.batching(8) == 0
    outs, tickets = [], []
    for i, g in enumerate(requests_):
        out = np.full(_nout(g), np.nan)
        geom = _host(g) if i % 2 == 0 else {k: torch.from_numpy(v).cuda() for k, v in _host(g).items()}
        tickets.append(srv.submit(g["kind"], geom, _load(g), out, opts=bie.make_opts(precision=bie.MIXED_FF)))
        outs.append(out)
    for t, out, ref in zip(tickets, outs, alone):
        rc, info, _ = srv.wait(t)
        assert rc == bie.OK
        assert info["rel_residual"] <= 1e-12
        assert _rel(out, ref) <= 1e-10
    batches = srv.batching()
    st = srv.stats()
    assert st["completed"] == len(requests_) and st["inflight_bytes"] == 0
    if cap:
        assert st["peak_inflight_bytes"] <= cap
    srv.close()
    print(f"cap {cap}: {batches} batched solves for {len(requests_)} requests")
    assert batches >= 1


def test_batching_bad_request_fails_alone(requests_, alone):
    srv = bie.Server(0, workers=1)
    srv.batching(16)
    opts = bie.make_opts(precision=bie.MIXED_FF)
    idx = [i for i, g in enumerate(requests_) if g["kind"] == 0][:5]
    g0 = requests_[idx[0]]
    bad = dict(_host(g0))
    bs = bad["body_start"].copy()
    bs = np.array([0, 3, bs[-1]], dtype=np.int32)  # a body of 3 nodes: invalid, found by the solve
    bad["body_start"] = bs
    # a long first request keeps the single worker busy while the rest queue
    first = synth.star_grid(seed=5, n=128, rows=4, cols=4)
    t_first = srv.submit(0, _host(first), synth.charges(16, np.random.default_rng(1)), np.empty(16), opts=opts)
    outs, tickets = [], []
    for k, i in enumerate(idx):
        g = requests_[i]
        out = np.empty(_nout(g))
        tickets.append(srv.submit(0, _host(g), _load(g), out, opts=opts))
        outs.append(out)
        if k == 1:
            tb = srv.submit(0, bad, np.zeros(2), np.empty(2), opts=opts)
            assert tb > 0
    assert srv.wait(t_first)[0] == bie.OK
    for t, out, i in zip(tickets, outs, idx):
        rc, _, _ = srv.wait(t)
        assert rc == bie.OK and _rel(out, alone[i]) <= 1e-10
    assert srv.wait(tb)[0] == bie.ERR_INVALID
    assert srv.batching() >= 1  # the requests behind the first one were taken together
    srv.close()
