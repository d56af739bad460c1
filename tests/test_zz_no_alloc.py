"""apply_operator_noalloc: the operator application for callers that cannot
allocate device memory (a fixed memory budget, a framework that owns every
allocation, or a loop that must not synchronise through cudaMalloc/cudaFree).

Its output must equal apply_operator's within the operator tolerances of the
parity tests (FP64: 1e-13; FP32 pair sums: the FP32 bound, since a different
source split regroups the FP32 tile sums; float-float: 1e-12), on two calls in
a row with different sizes, so that what an earlier call left in the shared
scratch array cannot leak into a later result.  It is also compared with the
FP64 oracle directly, and run once on a caller-made stream.
This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import geometry, laplace, stokes  # noqa: E402
from paper_1507_05925_gb300 import bie  # noqa: E402

pytestmark = pytest.mark.gpu

# as in test_gpu_parity: FP64, FP32 pair sums, float-float pair sums
TOL = {bie.FP64: {0: 1e-13, 1: 1e-13}, bie.MIXED: {0: 2e-6, 1: 5e-6}, bie.MIXED_FF: {0: 1e-12, 1: 1e-12}}


def _dev(g):
    out = {k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda() for k in ("x", "y", "dx", "dy", "ddx", "ddy")}
    out["body_start"] = torch.from_numpy(np.ascontiguousarray(g["body_start"])).cuda()
    return out


@pytest.mark.parametrize("kind", [bie.LAPLACE, bie.STOKES])
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED, bie.MIXED_FF])
def test_noalloc_matches_apply_operator(kind, prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05925_gb300 import build
    build.build()
    ctx = bie.Context(0)
    big = synth.star_grid(seed=3, rows=4, cols=5, n=200)                      # M = 4000
    small = synth.assemble([synth.ellipse(0, 0, 1.0, 0.5, 0.2, 137), synth.disc(3.0, 0.5, 0.8, 91)])
    rng = np.random.default_rng(9)
    for g in (big, small):  # two calls in a row; the second reuses a dirtier scratch
        gd = _dev(g)
        n = g["x"].size * (kind + 1)
        v = torch.from_numpy(rng.standard_normal(n)).cuda()
        ref = torch.empty(n, dtype=torch.float64, device="cuda")
        got = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        assert bie.apply_operator(ctx, gd, kind, prec, v, ref) == bie.OK
        assert bie.apply_operator_noalloc(gd, kind, prec, v, got) == bie.OK
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item() / ref.abs().max().item()
        assert err <= TOL[prec][kind], err
        # and against the FP64 oracle itself
        ora = (laplace if kind == 0 else stokes).apply(geometry.nodes(g), v.cpu().numpy())
        err_o = np.max(np.abs(got.cpu().numpy() - ora)) / np.max(np.abs(ora))
        assert err_o <= TOL[prec][kind], err_o
    ctx.close()


def test_noalloc_on_a_caller_stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05925_gb300 import build
    build.build()
    ctx = bie.Context(0)
    g = synth.star_grid(seed=5, rows=2, cols=3, n=160)
    gd = _dev(g)
    v = torch.from_numpy(np.random.default_rng(4).standard_normal(2 * g["x"].size)).cuda()
    ref = torch.empty_like(v)
    got = torch.full_like(v, float("nan"))
    assert bie.apply_operator(ctx, gd, bie.STOKES, bie.MIXED_FF, v, ref) == bie.OK
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        assert bie.apply_operator_noalloc(gd, bie.STOKES, bie.MIXED_FF, v, got, stream=st) == bie.OK
    st.synchronize()
    err = (got - ref).abs().max().item() / ref.abs().max().item()
    assert err <= TOL[bie.MIXED_FF][1], err
    ctx.close()


def test_noalloc_rejects_oversize_and_host_arrays():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = synth.assemble([synth.disc(3.0 * i, 0.0, 1.0, 8192) for i in range(3)])  # M = 24576 > 16384
    gd = _dev(g)
    v = torch.zeros(g["x"].size, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    assert bie.apply_operator_noalloc(gd, bie.LAPLACE, bie.FP64, v, out) == bie.ERR_NOMEM
    small = synth.assemble([synth.disc(0.0, 0.0, 1.0, 64)])
    host = {k: np.ascontiguousarray(small[k]) for k in ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")}
    assert bie.apply_operator_noalloc(host, bie.LAPLACE, bie.FP64, np.zeros(64), np.zeros(64)) == bie.ERR_INVALID
