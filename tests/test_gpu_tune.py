"""Autotuning of the pair-sum grid (bie_tune): the tuned split count keeps the
operator and the solves within their tolerances, and clearing the table
restores the occupancy rule's results bitwise."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import geometry, laplace, stokes  # noqa: E402
from paper_1507_05925_gb300 import bie  # noqa: E402
from test_gpu_parity import TOL32, TOL_SOLVE, multitile, ragged4, rel2, rel_max  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05925_gb300 import build
    build.build()
    c = bie.Context(0)
    yield c
    bie.tune_clear()
    c.close()


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("geo", ["ragged4", "multitile"])
def test_tuned_operator_within_tolerance(ctx, kind, geo):
    g = ragged4() if geo == "ragged4" else (multitile() if kind == 0 else multitile(rows=3, cols=3))
    M = g["x"].size
    v = np.random.default_rng(11).standard_normal(M * (kind + 1))
    before = np.empty_like(v)
    assert bie.apply_operator(ctx, g, kind, bie.MIXED, v, before) == bie.OK
    rc, S, ms = bie.tune(ctx, g, kind, bie.MIXED)
    assert rc == bie.OK and S >= 1 and ms > 0
    after = np.empty_like(v)
    assert bie.apply_operator(ctx, g, kind, bie.MIXED, v, after) == bie.OK
    ref = (laplace if kind == 0 else stokes).apply(geometry.nodes(g), v)
    assert rel_max(after, ref) <= TOL32[kind]
    bie.tune_clear()
    again = np.empty_like(v)
    assert bie.apply_operator(ctx, g, kind, bie.MIXED, v, again) == bie.OK
    assert np.array_equal(again, before)  # the occupancy rule's plan, same summation order
    print(f"{geo} kind={kind}: M={M} tuned splits {S}, {ms * 1e3:.1f} us")


def test_tuned_solve_matches_oracle(ctx):
    g = multitile()
    q = synth.charges(16, np.random.default_rng(12))
    for prec in (bie.MIXED, bie.MIXED_FF):
        assert bie.tune(ctx, g, 0, prec)[0] == bie.OK
    phi = np.empty(16)
    rc, info = bie.elastance_solve(ctx, g, q, phi, opts=bie.make_opts(precision=bie.MIXED_FF))
    assert rc == bie.OK
    assert rel2(phi, laplace.solve(g, q)["phi"]) <= TOL_SOLVE
    bie.tune_clear()


def test_install_given_split_count(ctx):
    g = ragged4()
    v = np.random.default_rng(13).standard_normal(g["x"].size)
    rc, S, ms = bie.tune(ctx, g, 0, bie.MIXED, splits=5)
    assert rc == bie.OK and S == 5 and ms == 0.0
    out = np.empty_like(v)
    assert bie.apply_operator(ctx, g, 0, bie.MIXED, v, out) == bie.OK
    assert rel_max(out, laplace.apply(geometry.nodes(g), v)) <= TOL32[0]
    bie.tune_clear()


def test_tune_rejects_bad_arguments(ctx):
    g = ragged4()
    assert bie.tune(ctx, g, 2, bie.MIXED)[0] == bie.ERR_INVALID
    assert bie.tune(ctx, g, 0, 7)[0] == bie.ERR_INVALID


def test_full_size_in_the_tuned_launch_configuration(ctx):
    # bench.py tunes the 100-star workload before timing it: the operator rows
    # and the solve in that launch configuration, against the oracle
    from test_gpu_parity import TOLFF, _check_full_size, _sampled_rows, to_dev
    g = synth.WORKLOADS["stars100_M25600"]()
    geo = geometry.nodes(g)
    gd = to_dev(g)
    splits = {prec: bie.tune(ctx, gd, 0, prec)[1] for prec in (bie.MIXED, bie.MIXED_FF)}
    print(f"tuned splits {splits}")
    M, N = geo["M"], geo["N"]
    v = np.random.default_rng(14).standard_normal(M)
    rows = np.unique(np.concatenate([np.random.default_rng(15).choice(M, 48, replace=False), [0, M - 1]]))
    ref = _sampled_rows(geo, 0, v, rows)
    for prec, tol in ((bie.MIXED, TOL32[0]), (bie.MIXED_FF, TOLFF)):
        out = torch.empty(M, dtype=torch.float64, device="cuda")
        assert bie.apply_operator(ctx, gd, 0, prec, torch.from_numpy(v).cuda(), out) == bie.OK
        assert rel_max(out.cpu().numpy()[rows], ref) <= tol
    q = torch.from_numpy(g["q"]).cuda()
    res = {}
    for prec in (bie.MIXED_FF, bie.MIXED, bie.FP64):
        phi = torch.empty(N, dtype=torch.float64, device="cuda")
        dens = torch.empty(M, dtype=torch.float64, device="cuda")
        rc, info = bie.elastance_solve(ctx, gd, q, phi, dens, opts=bie.make_opts(precision=prec))
        assert rc == bie.OK, info
        res[prec] = (phi.cpu().numpy(), dens.cpu().numpy(), info)
    for prec in (bie.MIXED_FF, bie.MIXED):
        phi, nu, info = res[prec]
        _check_full_size(g, geo, 0, phi, nu, info, res[bie.FP64][0])
    bie.tune_clear()
