"""Solves whose GMRES iterations are replayed as CUDA graphs, against the same
solves launched kernel by kernel.

On a stream that can be captured, one captured iteration is replayed in
chunks (the first as long as the last cycle of the same shape, so that few
iterations are launched after convergence; those return at once).  On the
legacy default stream nothing is captured.  Every kernel reduces in a fixed order, so the two
must agree bitwise, with the same iteration counts, and both must match the
FP64 oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import laplace, stokes  # noqa: E402
from paper_1507_05925_gb300 import bie  # noqa: E402
from test_gpu_parity import multitile, rel2, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-10


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05925_gb300 import build
    build.build()
    c = bie.Context(0)
    yield c
    c.close()


def _problem(kind, seed):
    g = multitile(seed=seed, rows=3, cols=3)
    N = g["body_start"].size - 1
    rng = np.random.default_rng(seed)
    if kind == 0:
        load = synth.charges(N, rng)
        return g, load, laplace.solve(g, load)["phi"]
    FT = synth.forces_torques(N, rng)
    return g, FT.reshape(-1), stokes.solve(g, FT)["UW"].reshape(-1)


def _solve(ctx, g, kind, load, stream, **opts):
    N = g["body_start"].size - 1
    out = torch.full((N if kind == 0 else 3 * N,), float("nan"), dtype=torch.float64, device="cuda")
    fn = bie.elastance_solve if kind == 0 else bie.mobility_solve
    rc, info = fn(ctx, to_dev(g), torch.from_numpy(np.ascontiguousarray(load)).cuda(), out,
                  opts=bie.make_opts(**opts), stream=stream)
    torch.cuda.synchronize()
    assert rc == bie.OK, (rc, ctx.last_error(), info)
    return info, out.cpu().numpy()


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED, bie.MIXED_FF])
def test_graph_replay_matches_kernel_by_kernel(ctx, kind, prec):
    g, load, ref = _problem(kind, 21 + kind)
    info0, out0 = _solve(ctx, g, kind, load, None, precision=prec)
    st = torch.cuda.Stream()
    for rep in range(2):  # the first call captures the iteration, the second sizes its chunks from the first
        info1, out1 = _solve(ctx, g, kind, load, st, precision=prec)
        print(f"kind={kind} prec={prec} rep={rep}: {info1}")
        assert np.array_equal(out0, out1)
        for key in ("iters", "refinements", "matvecs_fp64", "matvecs_fp32"):
            assert info0[key] == info1[key], (key, info0, info1)
        assert info0["graph_replay"] == 0 and info1["graph_replay"] == 1, (info0, info1)
    assert rel2(out1, ref) <= TOL_SOLVE


def test_graph_replay_with_fmm_and_restarts(ctx):
    # a short restart length makes every cycle end on the restart, not on convergence
    g, load, ref = _problem(1, 31)
    opts = dict(precision=bie.MIXED_FF, fmm_order=24, restart=6)
    info0, out0 = _solve(ctx, g, 1, load, None, **opts)
    info1, out1 = _solve(ctx, g, 1, load, torch.cuda.Stream(), **opts)
    assert np.array_equal(out0, out1)
    assert info0["iters"] == info1["iters"] and info0["iters"] > 6
    assert info1["graph_replay"] == 1
    assert rel2(out1, ref) <= TOL_SOLVE


def test_batched_graph_replay_matches(ctx):
    geoms = [synth.four_discs(seed=40 + i) for i in range(5)]
    loads = [synth.charges(4, np.random.default_rng(50 + i)) for i in range(5)]
    res = []
    bie.small_batch_path(0)  # the lockstep block-diagonal path, whose iteration is captured
    try:
        for stream in (None, torch.cuda.Stream()):
            outs = [torch.empty(4, dtype=torch.float64, device="cuda") for _ in geoms]
            rc, infos, status = bie.elastance_solve_batch(ctx, [to_dev(g) for g in geoms],
                                                          [torch.from_numpy(q).cuda() for q in loads], outs,
                                                          opts=bie.make_opts(precision=bie.MIXED_FF), stream=stream)
            torch.cuda.synchronize()
            assert rc == bie.OK, ctx.last_error()
            res.append([o.cpu().numpy() for o in outs])
            assert infos[0]["graph_replay"] == (0 if stream is None else 1)
    finally:
        bie.small_batch_path(1)
    for a, b, g, q in zip(res[0], res[1], geoms, loads):
        assert np.array_equal(a, b)
        assert rel2(b, laplace.solve(g, q)["phi"]) <= TOL_SOLVE


@pytest.mark.parametrize("kind", [0, 1])
def test_fmm_graphs_follow_the_tree(ctx, kind):
    """FMM solves replayed from captured graphs in one context while the tree
    changes: the same bodies translated (same sizes, another bounding square:
    the captured launches hold the square), then the tuned leaf population
    (another tree, reallocated buffers), then the first geometry again.  The
    solution is translation invariant, so every solve matches the oracle's
    solution of the first geometry, and each matches its kernel-by-kernel
    twin bitwise."""
    g, load, ref = _problem(kind, 43 + kind)
    h = dict(g)
    h["x"] = g["x"] + 7.3
    h["y"] = g["y"] - 2.1
    opts = dict(precision=bie.MIXED_FF, fmm_order=24)
    st = torch.cuda.Stream()
    for geo in (g, h, g):
        info1, out1 = _solve(ctx, geo, kind, load, st, **opts)
        info0, out0 = _solve(ctx, geo, kind, load, None, **opts)
        assert info1["graph_replay"] == 1
        assert np.array_equal(out0, out1)
        assert rel2(out1, ref) <= TOL_SOLVE
    gd = to_dev(h)
    try:
        rc, leaf, inner, ms = bie.tune_fmm(ctx, gd, kind, torch.from_numpy(np.ascontiguousarray(load)).cuda(),
                                           bie.make_opts(**opts), stream=st)
        assert rc == bie.OK, ctx.last_error()
        for geo in (h, g):
            info1, out1 = _solve(ctx, geo, kind, load, st, **opts)
            info0, out0 = _solve(ctx, geo, kind, load, None, **opts)
            assert np.array_equal(out0, out1)
            assert rel2(out1, ref) <= TOL_SOLVE
    finally:
        bie.tune_clear()
