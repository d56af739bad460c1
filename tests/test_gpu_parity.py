"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written here, derived in the design notes):
  FP64 operator           max |gpu - oracle| <= 1e-13 max |oracle|  (rounding order only)
  FP32-pair-sum operator  max |gpu - oracle| <= TOL32 max |oracle|
  float-float operator    max |gpu - oracle| <= TOLFF max |oracle|
  solves, all precisions  ||phi - phi_oracle|| / ||phi_oracle|| <= 1e-10 (same for (v, omega))
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import geometry, laplace, stokes  # noqa: E402
from paper_1507_05925_gb300 import bie  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-13
TOL32 = {0: 2e-6, 1: 5e-6}
TOLFF = 1e-12
TOL_OP = {bie.FP64: {0: TOL64, 1: TOL64}, bie.MIXED: TOL32, bie.MIXED_FF: {0: TOLFF, 1: TOLFF}}
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


def to_dev(g, device="cuda"):
    out = {k: torch.from_numpy(np.ascontiguousarray(g[k])).to(device)
           for k in ("x", "y", "dx", "dy", "ddx", "ddy")}
    out["body_start"] = torch.from_numpy(np.ascontiguousarray(g["body_start"])).to(device)
    if "interior_pt" in g:
        out["interior_pt"] = torch.from_numpy(np.ascontiguousarray(g["interior_pt"])).to(device)
    return out


def ragged4():
    return synth.assemble([synth.star(0, 0, 1.0, 0.25, 5, 0.3, 200), synth.ellipse(3.1, 0.2, 1.0, 0.45, 1.0, 137),
                           synth.disc(0.4, 3.0, 0.7, 91), synth.star(3.3, 3.2, 0.9, 0.2, 3, 1.3, 300)])


def multitile(seed=7, rows=4, cols=4):
    rng = np.random.default_rng(seed)
    curves = []
    for i in range(rows):
        for j in range(cols):
            n = int(rng.integers(64, 301))
            if (i + j) % 2:
                curves.append(synth.ellipse(3.2 * i, 3.2 * j, 1.0, rng.uniform(0.4, 1.0), rng.uniform(0, 3), n))
            else:
                curves.append(synth.star(3.2 * i, 3.2 * j, rng.uniform(0.6, 1.0), rng.uniform(0, 0.3),
                                         int(rng.integers(3, 7)), rng.uniform(0, 6), n))
    return synth.assemble(curves)


GEOMS = {"four_discs": lambda: synth.four_discs(seed=0), "ragged4": ragged4, "multitile": multitile}


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# operator parity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("kind", [bie.LAPLACE, bie.STOKES])
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED, bie.MIXED_FF])
def test_apply_operator(ctx, name, kind, prec):
    g = GEOMS[name]()
    if kind == bie.STOKES and name == "multitile":
        g = multitile(rows=3, cols=3)
    geo = geometry.nodes(g)
    n = geo["M"] * (kind + 1)
    v = np.random.default_rng(3).standard_normal(n)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = bie.apply_operator(ctx, to_dev(g), kind, prec, torch.from_numpy(v).cuda(), out)
    torch.cuda.synchronize()
    assert rc == bie.OK, ctx.last_error()
    ref = (laplace if kind == 0 else stokes).apply(geo, v)
    err = rel_max(out.cpu().numpy(), ref)
    tol = TOL_OP[prec][kind]
    print(f"apply {name} kind={kind} prec={prec}: rel max err {err:.2e}")
    assert err <= tol


# ---------------------------------------------------------------------------
# solve parity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED, bie.MIXED_FF])
@pytest.mark.parametrize("form", [0, 1])
def test_elastance_solve(ctx, name, prec, form):
    g = GEOMS[name]()
    N = g["body_start"].size - 1
    q = synth.charges(N, np.random.default_rng(11))
    ref = laplace.solve(g, q)
    phi = torch.empty(N, dtype=torch.float64, device="cuda")
    dens = torch.empty(g["x"].size, dtype=torch.float64, device="cuda")
    rc, info = bie.elastance_solve(ctx, to_dev(g), torch.from_numpy(q).cuda(), phi, dens,
                                   opts=bie.make_opts(precision=prec, formulation=form))
    torch.cuda.synchronize()
    assert rc == bie.OK, (rc, ctx.last_error(), info)
    e_phi = rel2(phi.cpu().numpy(), ref["phi"])
    w = ref["geo"]["w"]
    e_den = rel2(np.sqrt(w) * dens.cpu().numpy(), np.sqrt(w) * ref["nu"])
    print(f"elastance {name} prec={prec} form={form}: phi {e_phi:.2e} density {e_den:.2e} {info}")
    assert e_phi <= TOL_SOLVE
    assert e_den <= 1e-9
    assert info["rel_residual"] <= 1e-12
    assert info["constraint_residual"] <= 1e-10
    # the FP32 operator's measured error is reported by mixed solves only
    if prec == bie.FP64:
        assert info["fp32_error"] == 0.0
    else:
        assert 0.0 < info["fp32_error"] < TOL32[0]


@pytest.mark.parametrize("name", ["ragged4", "multitile"])
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED, bie.MIXED_FF])
@pytest.mark.parametrize("form", [0, 1])
def test_mobility_solve(ctx, name, prec, form):
    g = GEOMS[name]() if name == "ragged4" else multitile(rows=3, cols=3)
    N = g["body_start"].size - 1
    FT = synth.forces_torques(N, np.random.default_rng(12))
    ref = stokes.solve(g, FT)
    UW = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    dens = torch.empty(2 * g["x"].size, dtype=torch.float64, device="cuda")
    rc, info = bie.mobility_solve(ctx, to_dev(g), torch.from_numpy(FT.reshape(-1)).cuda(), UW, dens,
                                  opts=bie.make_opts(precision=prec, formulation=form))
    torch.cuda.synchronize()
    assert rc == bie.OK, (rc, ctx.last_error(), info)
    e = rel2(UW.cpu().numpy(), ref["UW"].reshape(-1))
    w2 = np.repeat(ref["geo"]["w"], 2)
    e_den = rel2(np.sqrt(w2) * dens.cpu().numpy(), np.sqrt(w2) * ref["nu"])
    print(f"mobility {name} prec={prec} form={form}: UW {e:.2e} density {e_den:.2e} {info}")
    assert e <= TOL_SOLVE
    assert e_den <= 1e-9
    assert info["rel_residual"] <= 1e-12


# ---------------------------------------------------------------------------
# block-Jacobi preconditioner of the inner solves: every inversion path
# (one CTA, clusters of four and eight CTAs, identity for large bodies)
# ---------------------------------------------------------------------------
def _precond_paths(kind):
    # unknowns per body: one CTA (<= 128), four-CTA cluster (<= 448),
    # eight-CTA cluster (<= 640), identity (> 640)
    n = (64, 200, 500, 700) if kind == 0 else (48, 150, 260, 330)
    curves = [synth.ellipse(0.0, 0.0, 1.0, 0.6, 0.3, n[0]), synth.star(3.0, 0.2, 1.0, 0.2, 5, 0.1, n[1]),
              synth.ellipse(0.3, 3.1, 1.2, 0.5, -0.4, n[2]), synth.star(3.4, 3.2, 1.1, 0.15, 3, 0.7, n[3])]
    return synth.assemble(curves)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("prec", [bie.MIXED, bie.MIXED_FF])
def test_block_jacobi_paths(ctx, kind, prec):
    g = _precond_paths(kind)
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
    infos = []
    for pc in (bie.PRECOND_BLOCK_JACOBI, bie.PRECOND_NONE):
        out = torch.empty(nout, dtype=torch.float64, device="cuda")
        rc, info = fn(ctx, to_dev(g), torch.from_numpy(load).cuda(), out,
                      opts=bie.make_opts(precision=prec, precond=pc))
        torch.cuda.synchronize()
        assert rc == bie.OK, (rc, ctx.last_error(), info)
        e = rel2(out.cpu().numpy(), ref)
        print(f"precond={pc} kind={kind} prec={prec}: {e:.2e} {info}")
        assert e <= TOL_SOLVE
        assert info["rel_residual"] <= 1e-12
        infos.append(info)
    # widely separated bodies: the blocks are well conditioned already, and the
    # preconditioner must not cost iterations
    assert infos[0]["matvecs_fp32"] <= infos[1]["matvecs_fp32"]


@pytest.mark.parametrize("wl,kind", [("stars100_M25600", 0), ("stars100_M25600", 1)])
def test_block_jacobi_cuts_inner_iterations(ctx, wl, kind):
    # 100 five- and three-armed stars: the self-interaction of each body is what
    # the unpreconditioned inner GMRES spends its iterations on
    g = synth.WORKLOADS[wl]()
    N = g["body_start"].size - 1
    if kind == 0:
        load, fn, nout = synth.charges(N, np.random.default_rng(23)), bie.elastance_solve, N
    else:
        load, fn, nout = synth.forces_torques(N, np.random.default_rng(24)).reshape(-1), bie.mobility_solve, 3 * N
    res, infos = [], []
    for pc in (bie.PRECOND_BLOCK_JACOBI, bie.PRECOND_NONE):
        out = torch.empty(nout, dtype=torch.float64, device="cuda")
        rc, info = fn(ctx, to_dev(g), torch.from_numpy(load).cuda(), out,
                      opts=bie.make_opts(precision=bie.MIXED_FF, precond=pc))
        torch.cuda.synchronize()
        assert rc == bie.OK, (rc, ctx.last_error(), info)
        print(f"{wl} kind={kind} precond={pc}: {info}")
        res.append(out.cpu().numpy())
        infos.append(info)
    assert rel2(res[0], res[1]) <= TOL_SOLVE
    assert infos[0]["matvecs_fp32"] < 0.75 * infos[1]["matvecs_fp32"]


def test_precond_option_validated(ctx):
    g = ragged4()
    N = g["body_start"].size - 1
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    rc, _ = bie.elastance_solve(ctx, to_dev(g), torch.zeros(N, dtype=torch.float64, device="cuda"), out,
                                opts=bie.make_opts(precision=bie.MIXED, precond=2))
    assert rc == bie.ERR_INVALID


# ---------------------------------------------------------------------------
# closed forms evaluated by the GPU path
# ---------------------------------------------------------------------------
def test_gpu_closed_forms(ctx):
    # single disc: phi = -(q/2pi) log R; single ellipse: -(q/2pi) log((a+b)/2)
    for curve, cap in ((synth.disc(0.3, -0.2, 1.7, 64), 1.7), (synth.ellipse(0.1, 0.2, 1.3, 0.4, 2.0, 256), 0.85)):
        g = synth.assemble([curve])
        phi = torch.empty(1, dtype=torch.float64, device="cuda")
        rc, _ = bie.elastance_solve(ctx, to_dev(g), torch.tensor([1.3], dtype=torch.float64, device="cuda"), phi)
        assert rc == bie.WARN_NONNEUTRAL  # a single charged conductor is not neutral
        assert abs(phi.item() + 1.3 / (2 * math.pi) * math.log(cap)) < 1e-13
    # two discs, gap 0.5: phi_1 - phi_2 = (Q/pi) log((alpha + d/2)/(alpha - d/2))
    d, Q = 0.5, 0.8
    g = synth.two_discs(d, 256)
    phi = torch.empty(2, dtype=torch.float64, device="cuda")
    rc, _ = bie.elastance_solve(ctx, to_dev(g), torch.tensor([Q, -Q], dtype=torch.float64, device="cuda"), phi,
                                opts=bie.make_opts(precision=bie.MIXED))
    al = math.sqrt(d + d * d / 4)
    p = phi.cpu().numpy()
    assert rc == bie.OK
    assert abs(p[0] - p[1] - Q / math.pi * math.log((al + d / 2) / (al - d / 2))) < 1e-12
    # rotating ellipse: omega = T / (2 pi (a^2 + b^2)); single disc translation
    g = synth.assemble([synth.ellipse(0.2, -0.1, 1.2, 0.3, 0.7, 256)])
    UW = torch.empty(3, dtype=torch.float64, device="cuda")
    rc, _ = bie.mobility_solve(ctx, to_dev(g), torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64, device="cuda"), UW)
    assert rc == bie.OK
    assert abs(UW[2].item() - 1.0 / (2 * math.pi * (1.44 + 0.09))) < 1e-13
    g = synth.assemble([synth.disc(0.3, -0.2, 1.7, 64)])
    rc, _ = bie.mobility_solve(ctx, to_dev(g), torch.tensor([0.7, -0.4, 1.1], dtype=torch.float64, device="cuda"), UW)
    assert rc == bie.WARN_NONNEUTRAL
    u = UW.cpu().numpy()
    # the solve stops at a relative residual of 1e-12; the single-layer sum that
    # gives v adds terms about 40 times v itself (|G| ~ 0.04 against v ~ 2e-3),
    # so the density's 1e-12 shows as up to ~1e-13 in v
    assert np.max(np.abs(u[:2] - np.array([0.7, -0.4]) * (0.5 - math.log(1.7)) / (4 * math.pi))) < 1e-13
    assert abs(u[2] - 1.1 / (4 * math.pi * 1.7**2)) < 1e-13


def test_two_disc_mobility_table_gpu(ctx):
    from conftest import read_golden
    kv, rows = read_golden("two_disc_mobility.txt")
    d, F11, F21, T1, T2 = rows[0][:5]
    FT = np.array([F11, F21, T1, -F11, -F21, T2])
    UW = torch.empty(6, dtype=torch.float64, device="cuda")
    rc, info = bie.mobility_solve(ctx, to_dev(synth.two_discs(d, 256)), torch.from_numpy(FT).cuda(), UW,
                                  opts=bie.make_opts(precision=bie.MIXED))
    assert rc == bie.OK
    u = UW.cpu().numpy().reshape(2, 3)
    assert np.max(np.abs((u[0, :2] - u[1, :2]) - np.array([2.09 - 1.00, -1.034 - 0.254]))) < 1e-5
    assert np.max(np.abs(u[:, 2] - np.array(kv["omega"]))) < 1e-5


# ---------------------------------------------------------------------------
# host pointers, determinism, edge cases
# ---------------------------------------------------------------------------
def test_host_and_device_pointers_agree_bitwise(ctx):
    g = ragged4()
    q = synth.charges(4, np.random.default_rng(5))
    phi_d = torch.empty(4, dtype=torch.float64, device="cuda")
    rc1, _ = bie.elastance_solve(ctx, to_dev(g), torch.from_numpy(q).cuda(), phi_d,
                                 opts=bie.make_opts(precision=bie.MIXED))
    phi_h = np.empty(4)
    host = {k: np.ascontiguousarray(g[k]) for k in ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")}
    rc2, _ = bie.elastance_solve(ctx, host, q, phi_h, opts=bie.make_opts(precision=bie.MIXED))
    torch.cuda.synchronize()
    assert rc1 == rc2 == bie.OK
    assert np.array_equal(phi_d.cpu().numpy(), phi_h)
    # repeat: identical bits (fixed-order reductions)
    phi_h2 = np.empty(4)
    bie.elastance_solve(ctx, host, q, phi_h2, opts=bie.make_opts(precision=bie.MIXED))
    assert np.array_equal(phi_h, phi_h2)


def test_minimum_size_and_interior_point(ctx):
    # 8 nodes (the minimum), user interior point off-centre
    g = synth.assemble([synth.disc(0.0, 0.0, 1.0, 8), synth.disc(3.0, 0.0, 1.0, 8)])
    g["interior_pt"] = np.array([0.2, 0.1, 3.1, -0.2])
    q = np.array([1.0, -1.0])
    phi = np.empty(2)
    rc, _ = bie.elastance_solve(ctx, g, q, phi)
    assert rc == bie.OK
    ref = laplace.solve(g, q)
    geo = ref["geo"]
    # the oracle's field at the same interior points
    u = laplace.single_layer_at(geo, ref["nu"], np.array([0.2, 3.1]), np.array([0.1, -0.2]))
    assert rel2(phi, u) < 1e-12


def test_invalid_arguments(ctx):
    g = ragged4()
    host = {k: np.ascontiguousarray(g[k]) for k in ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")}
    q = np.zeros(4)
    phi = np.empty(4)
    bad = dict(host, body_start=np.array([0, 200, 337, 340, 728], dtype=np.int32))  # body of 3 nodes
    assert bie.elastance_solve(ctx, bad, q, phi)[0] == bie.ERR_INVALID
    bad = dict(host, body_start=np.array([1, 200, 337, 428, 728], dtype=np.int32))
    assert bie.elastance_solve(ctx, bad, q, phi)[0] == bie.ERR_INVALID
    outside = dict(host, interior_pt=np.array([10.0, 10.0, 3.1, 0.2, 0.4, 3.0, 3.3, 3.2]))
    assert bie.elastance_solve(ctx, outside, q, phi)[0] == bie.ERR_OUTSIDE
    cw = {k: np.ascontiguousarray(v[::-1]) if k != "body_start" else v for k, v in
          synth.assemble([synth.disc(0, 0, 1, 32)]).items()}
    cw["dx"], cw["dy"] = -cw["dx"], -cw["dy"]
    assert bie.elastance_solve(ctx, cw, np.ones(1), np.empty(1))[0] == bie.ERR_OUTSIDE
    small = bie.Context(0, workspace_cap_bytes=1024)
    assert bie.elastance_solve(small, host, q, phi)[0] == bie.ERR_NOMEM
    small.close()
    rc, info = bie.elastance_solve(ctx, host, synth.charges(4, np.random.default_rng(1)), phi,
                                   opts=bie.make_opts(max_iter=2))
    assert rc == bie.WARN_NOT_CONVERGED and info["iters"] <= 2


def test_nonneutral_still_matches_oracle(ctx):
    g = ragged4()
    q = np.array([1.0, 0.5, -0.2, 0.3])
    phi = np.empty(4)
    rc, info = bie.elastance_solve(ctx, g, q, phi)
    assert rc == bie.WARN_NONNEUTRAL and abs(info["net_load"] - 1.6) < 1e-12
    assert rel2(phi, laplace.solve(g, q)["phi"]) <= TOL_SOLVE


# ---------------------------------------------------------------------------
# full-size workloads: sampled rows and size-independent properties
# ---------------------------------------------------------------------------
def _sampled_rows(geo, kind, v, rows):
    mod = laplace if kind == 0 else stokes
    A = mod.kernel_rows(geo, rows) + mod.completion_rows(geo, rows)
    if kind == 0:
        return 0.5 * v[rows] + A @ v
    idx = np.stack([2 * rows, 2 * rows + 1], 1).reshape(-1)
    return 0.5 * v[idx] + A @ v


@pytest.mark.parametrize("wl,kind", [("stars100_M25600", 0), ("ellipses400_M51200", 1)])
def test_full_size_operator_rows(ctx, wl, kind):
    g = synth.WORKLOADS[wl]()
    geo = geometry.nodes(g)
    n = geo["M"] * (kind + 1)
    v = np.random.default_rng(4).standard_normal(n)
    rows = np.sort(np.random.default_rng(5).choice(geo["M"], 48, replace=False))
    rows = np.unique(np.concatenate([rows, [0, geo["M"] - 1]]))
    ref = _sampled_rows(geo, kind, v, rows)
    gd = to_dev(g)
    for prec, tol in ((bie.FP64, TOL64), (bie.MIXED, TOL32[kind]), (bie.MIXED_FF, TOLFF)):
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        assert bie.apply_operator(ctx, gd, kind, prec, torch.from_numpy(v).cuda(), out) == bie.OK
        o = out.cpu().numpy()
        got = o[rows] if kind == 0 else o[np.stack([2 * rows, 2 * rows + 1], 1).reshape(-1)]
        err = rel_max(got, ref)
        print(f"{wl} rows prec={prec}: {err:.2e}")
        assert err <= tol


FULL_SIZE_GOLDEN = {"stars100_M25600": "stars100_M25600_elastance.txt",
                    "ellipses400_M51200": "ellipses400_M51200_mobility.txt"}


def _full_size_oracle(wl, g, load):
    """The oracle's solution of a full-size workload, stored by
    tests/golden/make_fullsize.py (dense LU for the 100 stars; GMRES on
    row-blocked operator applications to a true relative residual of 1e-13 for
    the 400 ellipses), after checking that the inputs are the ones it solved."""
    from conftest import read_golden
    kv, rows = read_golden(FULL_SIZE_GOLDEN[wl])
    assert int(kv["M"][0]) == g["x"].size and int(kv["N"][0]) == g["body_start"].size - 1
    for key, val in (("sum_x", np.sum(g["x"])), ("sum_y", np.sum(g["y"])), ("sum_load", np.sum(np.abs(load)))):
        assert abs(val - kv[key][0]) <= 1e-12 * abs(kv[key][0]), (key, val, kv[key][0])
    if "rel_residual" in kv:
        assert kv["rel_residual"][0] <= 1e-13
    return np.array(rows).reshape(-1)


@pytest.mark.parametrize("wl,kind", [("stars100_M25600", 0), ("ellipses400_M51200", 1)])
def test_full_size_solves_match_oracle(ctx, wl, kind):
    # the headline workloads, every precision, element by element against the
    # oracle's own solution of the same discrete system (eqs. ModRep2,
    # ModRep2Stokes), plus the sampled-row and constraint checks
    g = synth.WORKLOADS[wl]()
    geo = geometry.nodes(g)
    N, M = geo["N"], geo["M"]
    load = g["q"] if kind == 0 else g["FT"].reshape(-1)
    ref = _full_size_oracle(wl, g, load)
    gd = to_dev(g)
    outs = {}
    for prec in (bie.MIXED_FF, bie.MIXED, bie.FP64):
        out = torch.empty(N if kind == 0 else 3 * N, dtype=torch.float64, device="cuda")
        dens = torch.empty(M * (kind + 1), dtype=torch.float64, device="cuda")
        fn = bie.elastance_solve if kind == 0 else bie.mobility_solve
        rc, info = fn(ctx, gd, torch.from_numpy(load).cuda(), out, dens, opts=bie.make_opts(precision=prec))
        torch.cuda.synchronize()
        assert rc == bie.OK, (rc, info)
        res = out.cpu().numpy()
        e2, emax = rel2(res, ref), float(np.max(np.abs(res - ref)) / np.max(np.abs(ref)))
        print(f"{wl} prec={prec}: vs oracle rel2 {e2:.2e} relmax {emax:.2e} {info}")
        assert e2 <= TOL_SOLVE
        assert emax <= TOL_SOLVE
        outs[prec] = (res, dens.cpu().numpy(), info)
    for prec in (bie.MIXED, bie.MIXED_FF):
        res, nu, info = outs[prec]
        _check_full_size(g, geo, kind, res, nu, info, outs[bie.FP64][0])


@pytest.mark.parametrize("wl,kind", [("stars100_M25600", 0), ("stars100_M25600", 1), ("ellipses400_M51200", 1)])
def test_refinement_residual_is_certified(ctx, wl, kind):
    # the float-float refinement updates its residual with FP32 pair sums after
    # the first true residual; the reported relative residual (update plus its
    # error bound) must bound the true one, recomputed here with the FP64
    # operator from the returned density
    g = synth.WORKLOADS[wl]()
    geo = geometry.nodes(g)
    N, M = geo["N"], geo["M"]
    if kind == 0:
        load = g["q"]
    else:
        FT = g["FT"] if "FT" in g else synth.forces_torques(N, np.random.default_rng(25))
        load = FT.reshape(-1)
    gd = to_dev(g)
    out = torch.empty(N if kind == 0 else 3 * N, dtype=torch.float64, device="cuda")
    dens = torch.empty(M * (kind + 1), dtype=torch.float64, device="cuda")
    fn = bie.elastance_solve if kind == 0 else bie.mobility_solve
    rc, info = fn(ctx, gd, torch.from_numpy(load).cuda(), out, dens, opts=bie.make_opts(precision=bie.MIXED_FF))
    assert rc == bie.OK, (rc, info)
    Anu = torch.empty_like(dens)
    assert bie.apply_operator(ctx, gd, kind, bie.FP64, dens, Anu) == bie.OK
    torch.cuda.synchronize()
    if kind == 0:
        rhs = g["q"][geo["body"]]
        sw = np.sqrt(geo["w"])
    else:
        px, py = stokes.perp(geo)
        b = geo["body"]
        rhs = np.stack([FT[b, 0] + FT[b, 2] * px, FT[b, 1] + FT[b, 2] * py], 1).reshape(-1)
        sw = np.repeat(np.sqrt(geo["w"]), 2)
    true_rel = np.linalg.norm(sw * (Anu.cpu().numpy() - rhs)) / np.linalg.norm(sw * rhs)
    print(f"{wl} kind={kind}: reported {info['rel_residual']:.2e} true {true_rel:.2e} {info}")
    assert info["rel_residual"] <= 1e-12
    assert true_rel <= 1.5 * info["rel_residual"] + 1e-14
    assert 0.0 < info["fp32_error"] < TOL32[kind]


def _check_full_size(g, geo, kind, res, nu, info, res64):
    M = geo["M"]
    # (1) the density satisfies the oracle's equation at sampled rows: (1/2 I + K + L) nu = L sigma
    rows = np.sort(np.random.default_rng(6).choice(M, 40, replace=False))
    lhs = _sampled_rows(geo, kind, nu, rows)
    if kind == 0:
        rhs = g["q"][geo["body"][rows]]
    else:
        px, py = stokes.perp(geo)
        b = geo["body"][rows]
        FT = g["FT"]
        rhs = np.stack([FT[b, 0] + FT[b, 2] * px[rows], FT[b, 1] + FT[b, 2] * py[rows]], 1).reshape(-1)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-10
    # (2) the outputs recomputed by the oracle from the GPU density
    if kind == 0:
        ref = laplace.potentials_from_density(g, nu)
    else:
        ref = stokes.motion_from_density(g, nu).reshape(-1)
    assert rel2(res, ref) < 1e-12
    # (3) mixed precision and FP64 agree
    assert rel2(res, res64) < TOL_SOLVE
    # (4) constraints of the equivalence lemma
    assert info["constraint_residual"] < 1e-10


# ---------------------------------------------------------------------------
# the paper's round trip (Section 6.1) on the GPU path: charges from the
# capacitance oracle (a different integral equation) drive the GPU elastance
# solve, which must return the prescribed potentials minus the potential at
# infinity of the capacitance solution
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["four_discs", "ragged4", "multitile"])
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED, bie.MIXED_FF])
def test_capacitance_round_trip_on_gpu(ctx, name, prec):
    from oracle import capacitance
    g = GEOMS[name]()
    N = g["body_start"].size - 1
    phi = np.random.default_rng(31).standard_normal(N)
    cap = capacitance.solve(g, phi)
    out = np.empty(N)
    rc, info = bie.elastance_solve(ctx, g, cap["q"], out, opts=bie.make_opts(precision=prec))
    assert rc == bie.OK, (rc, info)
    back = out + cap["u_inf"]
    print(f"round trip {name} prec={prec}: {np.max(np.abs(back - phi)):.2e}")
    assert np.max(np.abs(back - phi)) <= 1e-10 * np.max(np.abs(phi))


@pytest.mark.parametrize("name", ["four_discs", "ragged4"])
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED, bie.MIXED_FF])
def test_resistance_round_trip_on_gpu(ctx, name, prec):
    # Section 6.2: forces and torques from the resistance oracle (a different
    # integral equation) drive the GPU mobility solve, which must return the
    # prescribed rigid motions less the velocity at infinity
    from oracle import resistance
    g = GEOMS[name]()
    N = g["body_start"].size - 1
    UW = np.random.default_rng(32).standard_normal((N, 3))
    res = resistance.solve(g, UW)
    out = np.empty(3 * N)
    rc, info = bie.mobility_solve(ctx, g, np.ascontiguousarray(res["FT"].reshape(-1)), out,
                                  opts=bie.make_opts(precision=prec))
    assert rc == bie.OK, (rc, info)
    target = UW.copy()
    target[:, :2] -= res["u_inf"]
    err = np.max(np.abs(out.reshape(N, 3) - target))
    print(f"mobility round trip {name} prec={prec}: {err:.2e}")
    assert err <= 1e-10 * np.max(np.abs(UW))


# ---------------------------------------------------------------------------
# the symmetric FP32 Laplace pair sum (the default plan once the 256-node tile
# pairs fill the GPU): ragged bodies, tiles that span bodies, a last partial
# tile, near and far tile pairs
# ---------------------------------------------------------------------------
def ragged_large(seed=31):
    rng = np.random.default_rng(seed)
    curves = []
    for i in range(8):
        for j in range(7):
            n = int(rng.integers(90, 331))
            if (i + j) % 3:
                curves.append(synth.ellipse(3.2 * i, 3.2 * j, 1.0, rng.uniform(0.4, 1.0), rng.uniform(0, 3), n))
            else:
                curves.append(synth.star(3.2 * i, 3.2 * j, rng.uniform(0.6, 1.0), rng.uniform(0, 0.3),
                                         int(rng.integers(3, 7)), rng.uniform(0, 6), n))
    return synth.assemble(curves)


def test_symmetric_pair_sum_operator_and_solve(ctx):
    g = ragged_large()
    geo = geometry.nodes(g)
    M = geo["M"]
    assert M % 256 != 0 and M > 9000
    gd = to_dev(g)
    v = np.random.default_rng(5).standard_normal(M)
    ref = laplace.apply(geo, v)
    bie.tune_clear()
    rc, S, _ = bie.tune(ctx, gd, bie.LAPLACE, bie.MIXED, splits=-1)  # the symmetric plan, explicitly
    assert rc == bie.OK and S == -((M + 255) // 256)
    out = torch.empty(M, dtype=torch.float64, device="cuda")
    assert bie.apply_operator(ctx, gd, bie.LAPLACE, bie.MIXED, torch.from_numpy(v).cuda(), out) == bie.OK
    torch.cuda.synchronize()
    sym = out.cpu().numpy()
    err = rel_max(sym, ref)
    print(f"symmetric FP32 Laplace operator, M={M}: {err:.2e}")
    assert err <= TOL32[0]
    # the directed kernel (a uniform split plan installed untimed) agrees
    rc, S, _ = bie.tune(ctx, gd, bie.LAPLACE, bie.MIXED, splits=24)
    assert rc == bie.OK and S > 0
    assert bie.apply_operator(ctx, gd, bie.LAPLACE, bie.MIXED, torch.from_numpy(v).cuda(), out) == bie.OK
    torch.cuda.synchronize()
    bie.tune_clear()
    # the symmetric plan is the occupancy rule's for this size; Stokes and FP64 have none
    assert bie.tune(ctx, gd, bie.STOKES, bie.MIXED, splits=-1)[0] == bie.ERR_INVALID
    assert bie.tune(ctx, gd, bie.LAPLACE, bie.FP64, splits=-1)[0] == bie.ERR_INVALID
    # the symmetric float-float kernel against the oracle (and the directed one)
    for S in (-1, 24):
        rc, SS, _ = bie.tune(ctx, gd, bie.LAPLACE, bie.MIXED_FF, splits=S)
        assert rc == bie.OK and (SS < 0) == (S < 0)
        assert bie.apply_operator(ctx, gd, bie.LAPLACE, bie.MIXED_FF, torch.from_numpy(v).cuda(), out) == bie.OK
        torch.cuda.synchronize()
        e = rel_max(out.cpu().numpy(), ref)
        print(f"float-float Laplace operator, plan {SS}: {e:.2e}")
        assert e <= TOLFF
    bie.tune_clear()
    assert rel_max(out.cpu().numpy(), ref) <= TOL32[0]
    assert rel_max(out.cpu().numpy(), sym) <= 2 * TOL32[0]
    # a mixed-precision solve on the symmetric kernel, against the oracle's LU
    N = geo["N"]
    q = synth.charges(N, np.random.default_rng(12))
    phi_ref = laplace.solve(g, q)["phi"]
    for prec in (bie.MIXED, bie.MIXED_FF):
        phi = torch.empty(N, dtype=torch.float64, device="cuda")
        rc, info = bie.elastance_solve(ctx, gd, torch.from_numpy(q).cuda(), phi, opts=bie.make_opts(precision=prec))
        torch.cuda.synchronize()
        assert rc == bie.OK, (rc, ctx.last_error(), info)
        assert rel2(phi.cpu().numpy(), phi_ref) <= TOL_SOLVE


def test_output_logarithm_against_library(ctx):
    """The table-driven FP64 logarithm of the output sums (Tang 1990) against
    the CUDA library's log over 24 decades, near 1, at powers of two and at
    the special values: within 2 ulp of the result plus 4 * 2^-53 absolute
    (the cancellation of e log 2 against log c for x just below 1 costs
    relative, not absolute, accuracy; the sums need absolute accuracy)."""
    rng = np.random.default_rng(77)
    x = np.concatenate([10.0 ** rng.uniform(-12, 12, 200000), 1.0 + rng.uniform(-1e-3, 1e-3, 20000),
                        2.0 ** np.arange(-60, 61), 1.0 + (np.arange(128) + 0.5) / 128,
                        [1e-300, 1e300, 3.0, 0.0, 1e-310, np.inf]])
    xt = torch.from_numpy(x).cuda()
    out = torch.empty(2 * x.size, dtype=torch.float64, device="cuda")
    assert bie.test_log(xt, out) == bie.OK
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    a, b = o[:x.size], o[x.size:]
    fin = np.isfinite(b)
    assert np.array_equal(a[~fin], b[~fin])  # log 0 = -inf, log inf = inf: the library's values
    err = np.abs(a[fin] - b[fin])
    bound = 2 * np.spacing(np.abs(b[fin])) + 4 * 2.0 ** -53
    print(f"table log: max |diff| {err.max():.2e}, max diff / ulp {np.max(err / np.spacing(np.abs(b[fin]))):.2f}")
    assert np.all(err <= bound)
