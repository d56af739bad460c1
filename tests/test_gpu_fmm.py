"""Quadtree FMM pair sums: operator parity with the direct FP64 sums and the
oracle, determinism, and solves with FMM pair sums against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import geometry, laplace, stokes  # noqa: E402
from paper_1507_05925_gb300 import bie  # noqa: E402
from test_gpu_parity import _sampled_rows, multitile, rel2, rel_max, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

# FMM order -> operator tolerance (relative max-norm): the truncation decays
# about like 0.35^p for the 3 x 3-neighbour separation of this quadtree
TOL_FMM = {16: 1e-6, 36: 1e-12}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05925_gb300 import build
    build.build()
    c = bie.Context(0)
    yield c
    c.close()


def _apply(ctx, g, kind, v, order=None, prec=bie.FP64):
    out = torch.empty(v.size, dtype=torch.float64, device="cuda")
    vin = torch.from_numpy(v).cuda()
    if order is None:
        rc = bie.apply_operator(ctx, to_dev(g), kind, prec, vin, out)
    else:
        rc = bie.apply_operator_fmm(ctx, to_dev(g), kind, order, vin, out)
    torch.cuda.synchronize()
    assert rc == bie.OK, ctx.last_error()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", [bie.LAPLACE, bie.STOKES])
@pytest.mark.parametrize("order", [16, 36])
def test_fmm_operator_matches_direct(ctx, kind, order):
    g = multitile(rows=5, cols=5)
    v = np.random.default_rng(3).standard_normal(g["x"].size * (kind + 1))
    ref = _apply(ctx, g, kind, v)
    got = _apply(ctx, g, kind, v, order=order)
    err = rel_max(got, ref)
    print(f"fmm kind={kind} order={order}: {err:.2e}")
    assert err <= TOL_FMM[order]
    assert np.array_equal(got, _apply(ctx, g, kind, v, order=order))  # deterministic


def _apply_prec(ctx, g, kind, v, order, prec):
    out = torch.empty(v.size, dtype=torch.float64, device="cuda")
    rc = bie.apply_operator_fmm_prec(ctx, to_dev(g), kind, order, prec, torch.from_numpy(v).cuda(), out)
    torch.cuda.synchronize()
    assert rc == bie.OK, ctx.last_error()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", [bie.LAPLACE, bie.STOKES])
def test_fmm_operator_in_solve_precisions(ctx, kind):
    """The FMM operator as the solves use it: the inner solves' FP32 expansions
    (order 18) and the float-float refinement's residual operator (order 36,
    float-float multipole-to-local step), against the direct FP64 sums; the
    float-float one also against the FP64-expansion FMM, which isolates its
    rounding (about 2^-48 a step) from the truncation of the expansions."""
    g = multitile(rows=5, cols=5)
    v = np.random.default_rng(13).standard_normal(g["x"].size * (kind + 1))
    ref = _apply(ctx, g, kind, v)
    got32 = _apply_prec(ctx, g, kind, v, 18, bie.MIXED)
    gotff = _apply_prec(ctx, g, kind, v, 36, bie.MIXED_FF)
    fmm64 = _apply(ctx, g, kind, v, order=36)
    e32, eff, eff64 = rel_max(got32, ref), rel_max(gotff, ref), rel_max(gotff, fmm64)
    print(f"kind={kind}: fp32 expansions {e32:.2e}, float-float M2L {eff:.2e} (vs FP64 FMM {eff64:.2e})")
    assert e32 <= 2e-5
    assert eff <= TOL_FMM[36]
    assert eff64 <= 1e-13
    assert np.array_equal(gotff, _apply_prec(ctx, g, kind, v, 36, bie.MIXED_FF))  # deterministic
    assert bie.apply_operator_fmm_prec(ctx, to_dev(g), kind, 36, 7, torch.from_numpy(v).cuda(),
                                       torch.empty(v.size, dtype=torch.float64, device="cuda")) == bie.ERR_INVALID


@pytest.mark.parametrize("wl,kind,nrows", [("stars100_M25600", 0, 48), ("ellipses400_M51200", 1, 24),
                                           ("ellipses10000_M640000", 1, 8)])
def test_fmm_full_size_rows(ctx, wl, kind, nrows):
    g = synth.WORKLOADS[wl]()
    geo = geometry.nodes(g)
    v = np.random.default_rng(4).standard_normal(geo["M"] * (kind + 1))
    rows = np.sort(np.random.default_rng(5).choice(geo["M"], nrows, replace=False))
    ref = _sampled_rows(geo, kind, v, rows)
    got = _apply(ctx, g, kind, v, order=36)
    got = got[rows] if kind == 0 else got[np.stack([2 * rows, 2 * rows + 1], 1).reshape(-1)]
    err = rel_max(got, ref)
    print(f"fmm {wl} rows: {err:.2e}")
    assert err <= TOL_FMM[36]


@pytest.mark.parametrize("kind", [bie.LAPLACE, bie.STOKES])
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED_FF])
def test_solve_with_fmm(ctx, kind, prec):
    g = multitile(rows=4, cols=4) if kind == 0 else multitile(rows=3, cols=3)
    N = g["body_start"].size - 1
    if kind == 0:
        load = synth.charges(N, np.random.default_rng(11))
        ref = laplace.solve(g, load)["phi"]
        out = torch.empty(N, dtype=torch.float64, device="cuda")
        fn = bie.elastance_solve
    else:
        FT = synth.forces_torques(N, np.random.default_rng(12))
        load = FT.reshape(-1)
        ref = stokes.solve(g, FT)["UW"].reshape(-1)
        out = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        fn = bie.mobility_solve
    rc, info = fn(ctx, to_dev(g), torch.from_numpy(load).cuda(), out,
                  opts=bie.make_opts(precision=prec, fmm_order=36))
    torch.cuda.synchronize()
    assert rc == bie.OK, (rc, ctx.last_error(), info)
    err = rel2(out.cpu().numpy(), ref)
    print(f"fmm solve kind={kind} prec={prec}: {err:.2e} {info}")
    assert err <= 1e-10
    assert info["rel_residual"] <= 1e-12


def test_large_mobility_solve_with_fmm(ctx):
    # 10,000 ellipses x 64 nodes: FMM pair sums and FMM output evaluation
    g = synth.WORKLOADS["ellipses10000_M640000"]()
    geo = geometry.nodes(g)
    N, M = geo["N"], geo["M"]
    UW = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    dens = torch.empty(2 * M, dtype=torch.float64, device="cuda")
    rc, info = bie.mobility_solve(ctx, to_dev(g), torch.from_numpy(g["FT"].reshape(-1)).cuda(), UW, dens,
                                  opts=bie.make_opts(precision=bie.MIXED_FF, fmm_order=36))
    torch.cuda.synchronize()
    assert rc == bie.OK, (rc, ctx.last_error(), info)
    print(f"large mobility: {info}")
    nu = dens.cpu().numpy()
    res = UW.cpu().numpy().reshape(N, 3)
    # (1) outputs at 20 sampled bodies recomputed by the oracle from the density
    pts = geometry.interior_points(geo)
    idx = np.sort(np.random.default_rng(8).choice(N, 20, replace=False))
    z0x, z0y, d = pts["z0x"][idx], pts["z0y"][idx], pts["delta"][idx]
    u0 = stokes.single_layer_at(geo, nu, z0x, z0y)
    u1 = stokes.single_layer_at(geo, nu, z0x + d, z0y)
    u2 = stokes.single_layer_at(geo, nu, z0x, z0y + d)
    om = ((u1[:, 1] - u0[:, 1]) - (u2[:, 0] - u0[:, 0])) / (2 * d)
    ref = np.stack([u0[:, 0], u0[:, 1], om], 1)
    assert rel2(res[idx], ref) < 1e-11
    # (2) the density satisfies the oracle's equation at sampled rows
    rows = np.sort(np.random.default_rng(9).choice(M, 8, replace=False))
    lhs = _sampled_rows(geo, 1, nu, rows)
    px, py = stokes.perp(geo)
    b = geo["body"][rows]
    FT = g["FT"]
    rhs = np.stack([FT[b, 0] + FT[b, 2] * px[rows], FT[b, 1] + FT[b, 2] * py[rows]], 1).reshape(-1)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-10
    assert info["rel_residual"] <= 1e-12


@pytest.mark.parametrize("kind", [bie.LAPLACE, bie.STOKES])
def test_tuned_fmm_schedule_keeps_the_solution(ctx, kind):
    # bie_tune_fmm times whole solves over leaf populations and inner orders;
    # whatever it keeps, the solve still matches the oracle
    g = multitile(rows=4, cols=4) if kind == 0 else multitile(rows=3, cols=3)
    N = g["body_start"].size - 1
    if kind == 0:
        load = synth.charges(N, np.random.default_rng(21))
        ref = laplace.solve(g, load)["phi"]
        fn, nout = bie.elastance_solve, N
    else:
        FT = synth.forces_torques(N, np.random.default_rng(22))
        load = FT.reshape(-1)
        ref = stokes.solve(g, FT)["UW"].reshape(-1)
        fn, nout = bie.mobility_solve, 3 * N
    opts = bie.make_opts(precision=bie.MIXED_FF, fmm_order=24)
    gd = to_dev(g)
    ld = torch.from_numpy(load).cuda()
    try:
        rc, leaf, inner, ms = bie.tune_fmm(ctx, gd, kind, ld, opts)
        assert rc == bie.OK, ctx.last_error()
        assert leaf in (12, 24, 48) and 2 <= inner <= 24 and ms > 0
        out = torch.empty(nout, dtype=torch.float64, device="cuda")
        rc, info = fn(ctx, gd, ld, out, opts=opts)
        torch.cuda.synchronize()
        assert rc == bie.OK, (rc, ctx.last_error(), info)
        print(f"tuned fmm kind={kind}: leaf {leaf} inner {inner} {ms:.3f} ms {info}")
        assert rel2(out.cpu().numpy(), ref) <= 1e-10
    finally:
        bie.tune_clear()
    # invalid requests are refused
    assert bie.tune_fmm(ctx, gd, kind, ld, bie.make_opts(precision=bie.MIXED_FF))[0] == bie.ERR_INVALID
    assert bie.tune_fmm(ctx, gd, kind, ld, bie.make_opts(precision=bie.FP64, fmm_order=24))[0] == bie.ERR_INVALID


@pytest.mark.parametrize("kind", [bie.LAPLACE, bie.STOKES])
@pytest.mark.parametrize("prec", [bie.MIXED, bie.MIXED_FF])
def test_fmm_residuals_only(ctx, kind, prec):
    """fmm_order = -p: direct FP32 pair sums in the inner solves, the FMM of
    order p for the refinement's residuals and the output sums; against the
    oracle, and refused for FP64 GMRES."""
    g = multitile(rows=4, cols=4) if kind == 0 else multitile(rows=3, cols=3)
    N = g["body_start"].size - 1
    if kind == 0:
        load = synth.charges(N, np.random.default_rng(21))
        ref = laplace.solve(g, load)["phi"]
        fn, nout = bie.elastance_solve, N
    else:
        FT = synth.forces_torques(N, np.random.default_rng(22))
        load = FT.reshape(-1)
        ref = stokes.solve(g, FT)["UW"].reshape(-1)
        fn, nout = bie.mobility_solve, 3 * N
    out = torch.empty(nout, dtype=torch.float64, device="cuda")
    rc, info = fn(ctx, to_dev(g), torch.from_numpy(load).cuda(), out,
                  opts=bie.make_opts(precision=prec, fmm_order=-36))
    torch.cuda.synchronize()
    assert rc == bie.OK, (rc, ctx.last_error(), info)
    err = rel2(out.cpu().numpy(), ref)
    print(f"fmm residuals only kind={kind} prec={prec}: {err:.2e} {info}")
    assert err <= 1e-10
    assert info["rel_residual"] <= 1e-12 and info["matvecs_fp32"] > 0
    rc, _ = fn(ctx, to_dev(g), torch.from_numpy(load).cuda(), out, opts=bie.make_opts(precision=bie.FP64, fmm_order=-36))
    assert rc == bie.ERR_INVALID
    rc, _ = fn(ctx, to_dev(g), torch.from_numpy(load).cuda(), out, opts=bie.make_opts(precision=prec, fmm_order=-70))
    assert rc == bie.ERR_INVALID
