"""Batched solves: many independent problems solved as one block-diagonal
system must give each problem its own solution (oracle and solo solves), with
no pair or output sum crossing between problems."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import laplace, stokes  # noqa: E402
from paper_1507_05925_gb300 import bie  # noqa: E402
from test_gpu_parity import TOL_SOLVE, rel2  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05925_gb300 import build
    build.build()
    c = bie.Context(0)
    yield c
    c.close()


def _host(g):
    return {k: np.ascontiguousarray(g[k]) for k in ("x", "y", "dx", "dy", "ddx", "ddy", "body_start")}


def _problems(kind, seed, count):
    # ragged: 1-8 bodies of 40-200 nodes, so target blocks straddle problems
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        g = synth.random_request(rng, max_bodies=8, nodes=(40, 64, 137, 200))
        N = g["body_start"].size - 1
        if kind == 0:
            load = synth.charges(N, rng)
        else:
            load = synth.forces_torques(N, rng).reshape(-1)
        out.append((g, np.ascontiguousarray(load)))
    return out


def _oracle(kind, g, load):
    if kind == 0:
        return laplace.solve(g, load)["phi"]
    return stokes.solve(g, load.reshape(-1, 3))["UW"].reshape(-1)


def _solve_batch(ctx, kind, probs, opts, device=False):
    geoms = [_host(g) for g, _ in probs]
    loads = [ld for _, ld in probs]
    outs = [np.full(ld.size, np.nan) for ld in loads]
    if device:
        geoms = [{k: torch.from_numpy(v).cuda() for k, v in gm.items()} for gm in geoms]
        loads = [torch.from_numpy(ld).cuda() for ld in loads]
        outs = [torch.full((ld.shape[0],), float("nan"), dtype=torch.float64, device="cuda") for ld in loads]
    fn = bie.elastance_solve_batch if kind == 0 else bie.mobility_solve_batch
    rc, infos, status = fn(ctx, geoms, loads, outs, opts=opts)
    torch.cuda.synchronize()
    assert len(infos) == len(status) == len(probs)
    if rc >= 0:
        # the batch's status is the worst of the problems' own
        worst = bie.WARN_NOT_CONVERGED if bie.WARN_NOT_CONVERGED in status else max(status)
        assert rc == worst
    return rc, infos, status, [o.cpu().numpy() if device else o for o in outs]


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED, bie.MIXED_FF])
def test_batch_matches_oracle_and_solo(ctx, kind, prec):
    probs = _problems(kind, 50 + kind, 7)
    opts = bie.make_opts(precision=prec)
    rc, infos, status, outs = _solve_batch(ctx, kind, probs, opts, device=(prec == bie.MIXED))
    assert rc == bie.OK, (rc, ctx.last_error(), infos)
    assert status == [bie.OK] * len(probs)
    fn = bie.elastance_solve if kind == 0 else bie.mobility_solve
    for (g, load), out, info in zip(probs, outs, infos):
        assert info["rel_residual"] <= 1e-12
        ref = _oracle(kind, g, load)
        assert rel2(out, ref) <= TOL_SOLVE
        solo = np.empty_like(out)
        rc1, info1 = fn(ctx, _host(g), load, solo, opts=opts)
        assert rc1 == bie.OK
        assert rel2(out, solo) <= TOL_SOLVE
        # per-problem constraint residual and net load are the problem's own
        assert info["net_load"] == pytest.approx(info1["net_load"], abs=1e-13)
        assert info["constraint_residual"] <= 1e-6
    print(f"batch kind={kind} prec={prec}: {infos[0]}")


@pytest.mark.parametrize("kind", [0, 1])
def test_overlapping_problems_do_not_interact(ctx, kind):
    # the same geometry 9 times at the same place with different loads: any
    # pair crossing problems would couple them
    g = synth.four_discs(seed=3, n=128)
    rng = np.random.default_rng(60)
    probs = []
    for _ in range(9):
        load = synth.charges(4, rng) if kind == 0 else synth.forces_torques(4, rng).reshape(-1)
        probs.append((g, np.ascontiguousarray(load)))
    rc, _, _, outs = _solve_batch(ctx, kind, probs, bie.make_opts(precision=bie.MIXED_FF))
    assert rc == bie.OK, (rc, ctx.last_error())
    for (gg, load), out in zip(probs, outs):
        assert rel2(out, _oracle(kind, gg, load)) <= TOL_SOLVE


def test_batch_of_one_equals_solo(ctx):
    (g, load), = _problems(0, 70, 1)
    rc, _, _, outs = _solve_batch(ctx, 0, [(g, load)], bie.make_opts(precision=bie.MIXED_FF))
    assert rc == bie.OK, ctx.last_error()
    solo = np.empty(load.size)
    assert bie.elastance_solve(ctx, _host(g), load, solo, opts=bie.make_opts(precision=bie.MIXED_FF))[0] == bie.OK
    assert rc == bie.OK and rel2(outs[0], solo) <= TOL_SOLVE


def test_batch_nonneutral_and_errors(ctx):
    probs = _problems(0, 80, 3)
    g, load = probs[1]
    probs[1] = (g, load + 1.0)  # one charged problem among neutral ones
    rc, infos, status, outs = _solve_batch(ctx, 0, probs, bie.make_opts(precision=bie.MIXED_FF))
    assert rc == bie.WARN_NONNEUTRAL
    assert status == [bie.OK, bie.WARN_NONNEUTRAL, bie.OK]  # only the charged problem warns
    assert infos[1]["net_load"] == pytest.approx(abs(float(np.sum(load + 1.0))), rel=1e-12)
    assert infos[0]["net_load"] < 1e-12
    assert rel2(outs[1], _oracle(0, g, load + 1.0)) <= TOL_SOLVE
    geoms = [_host(gg) for gg, _ in probs]
    loads = [ld for _, ld in probs]
    outs = [np.empty(ld.size) for ld in loads]
    assert bie.elastance_solve_batch(ctx, geoms, loads, outs, opts=bie.make_opts(fmm_order=16))[0] == bie.ERR_INVALID
    bad = dict(geoms[2])
    bad["body_start"] = bad["body_start"].copy()
    bad["body_start"][1] = 3  # a body of 3 nodes
    assert bie.elastance_solve_batch(ctx, [geoms[0], bad], loads[:2], outs[:2])[0] == bie.ERR_INVALID
    assert "fewer than 8" in ctx.last_error()


@pytest.mark.parametrize("prec", [bie.FP64, bie.MIXED_FF])
def test_zero_load_problem_in_batch(ctx, prec):
    probs = _problems(1, 90, 4)
    g, load = probs[2]
    probs[2] = (g, np.zeros_like(load))
    rc, _, _, outs = _solve_batch(ctx, 1, probs, bie.make_opts(precision=prec))
    assert rc == bie.OK, ctx.last_error()
    assert np.all(outs[2] == 0.0)
    for i in (0, 1, 3):
        assert rel2(outs[i], _oracle(1, *probs[i])) <= TOL_SOLVE


@pytest.mark.parametrize("kind", [0, 1])
def test_batch_iterations_follow_the_slowest_problem(ctx, kind):
    # one Krylov space per problem: the lockstep count is about the slowest
    # problem's own count, not more because the problems are many
    rng = np.random.default_rng(95)
    probs = []
    for i in range(32):
        g = synth.four_discs(seed=i)
        load = synth.charges(4, rng) if kind == 0 else synth.forces_torques(4, rng).reshape(-1)
        probs.append((g, np.ascontiguousarray(load)))
    bie.small_batch_path(False)  # the lockstep multi-launch path (small batches default to one launch)
    try:
        _lockstep_iterations(ctx, kind, probs)
    finally:
        bie.small_batch_path(True)


def _lockstep_iterations(ctx, kind, probs):
    for prec in (bie.FP64, bie.MIXED_FF):
        opts = bie.make_opts(precision=prec)
        rc, infos, _, outs = _solve_batch(ctx, kind, probs, opts)
        assert rc == bie.OK
        info = infos[0]
        fn = bie.elastance_solve if kind == 0 else bie.mobility_solve
        solo_iters = []
        for (g, load), out in zip(probs, outs):
            solo = np.empty_like(out)
            rc1, inf1 = fn(ctx, _host(g), load, solo, opts=opts)
            assert rc1 == bie.OK
            solo_iters.append(inf1["iters"])
            assert rel2(out, solo) <= TOL_SOLVE
        print(f"kind={kind} prec={prec} batch iters {info['iters']} solo max {max(solo_iters)} "
              f"rel_residual {max(i['rel_residual'] for i in infos):.2e}")
        assert info["iters"] <= max(solo_iters) + 2
        assert max(i["rel_residual"] for i in infos) <= 1e-12


@pytest.mark.parametrize("kind", [0, 1])
def test_batch_mixed_host_and_device_arrays(ctx, kind):
    # staging gathers device arrays in one launch and packs host arrays: any mix
    # of the two, also within one problem, gives the same results
    probs = _problems(kind, 120 + kind, 6)
    opts = bie.make_opts(precision=bie.MIXED_FF)
    ref = _solve_batch(ctx, kind, probs, opts)[3]
    geoms, loads, outs = [], [], []
    for i, (g, load) in enumerate(probs):
        h = _host(g)
        if i % 3 == 0:
            gm = h
        elif i % 3 == 1:
            gm = {k: torch.from_numpy(v).cuda() for k, v in h.items()}
        else:  # body_start and positions on the device, derivatives on the host
            gm = {k: (torch.from_numpy(v).cuda() if k in ("body_start", "x", "y") else v) for k, v in h.items()}
        geoms.append(gm)
        loads.append(load if i % 2 == 0 else torch.from_numpy(load).cuda())
        outs.append(np.empty(load.size) if i % 2 == 1 else torch.empty(load.size, dtype=torch.float64, device="cuda"))
    fn = bie.elastance_solve_batch if kind == 0 else bie.mobility_solve_batch
    rc, _, status = fn(ctx, geoms, loads, outs, opts=opts)
    torch.cuda.synchronize()
    assert rc == bie.OK and status == [bie.OK] * len(probs)
    for out, r in zip(outs, ref):
        o = out.cpu().numpy() if isinstance(out, torch.Tensor) else out
        assert np.array_equal(o, r)  # staging does not change the arithmetic


def _with_points(g, shift):
    # one interior point per body: the mean of its nodes, shifted a little
    bs = g["body_start"]
    pts = []
    for i in range(bs.size - 1):
        pts += [g["x"][bs[i]:bs[i + 1]].mean() + shift, g["y"][bs[i]:bs[i + 1]].mean() - shift]
    h = _host(g)
    h["interior_pt"] = np.array(pts)
    return h


def test_batch_interior_points(ctx):
    probs = _problems(0, 140, 4)
    opts = bie.make_opts(precision=bie.MIXED_FF)
    geoms = [_with_points(g, 0.05) for g, _ in probs]
    loads = [ld for _, ld in probs]
    outs = [np.empty(ld.size) for ld in loads]
    rc, _, status = bie.elastance_solve_batch(ctx, geoms, loads, outs, opts=opts)
    assert rc == bie.OK and status == [bie.OK] * 4
    for gm, ld, out in zip(geoms, loads, outs):
        solo = np.empty_like(out)
        assert bie.elastance_solve(ctx, gm, ld, solo, opts=opts)[0] == bie.OK
        # (a single body's neutral charge is zero: both results are zero)
        assert np.linalg.norm(out - solo) <= TOL_SOLVE * np.linalg.norm(solo) + 1e-15
    # interior points for all problems or for none; a point outside its body
    mixed = [geoms[0], _host(probs[1][0])]
    assert bie.elastance_solve_batch(ctx, mixed, loads[:2], outs[:2], opts=opts)[0] == bie.ERR_INVALID
    bad = dict(geoms[2])
    bad["interior_pt"] = bad["interior_pt"].copy()
    bad["interior_pt"][:2] = [1e3, 1e3]
    assert bie.elastance_solve_batch(ctx, [geoms[0], bad], loads[:2], outs[:2], opts=opts)[0] == bie.ERR_OUTSIDE


@pytest.mark.parametrize("kind", [0, 1])
def test_batch_of_many_small_problems(ctx, kind):
    # more problems than the batched Arnoldi step has CTAs: ranges per CTA > 1
    rng = np.random.default_rng(150 + kind)
    probs = []
    for i in range(700):
        g = synth.assemble([synth.disc(0.0, 0.0, rng.uniform(0.5, 1.0), 16),
                            synth.ellipse(3.0, rng.uniform(-0.3, 0.3), 1.0, rng.uniform(0.4, 1.0), rng.uniform(0, 3), 16)])
        load = synth.charges(2, rng) if kind == 0 else synth.forces_torques(2, rng).reshape(-1)
        probs.append((g, np.ascontiguousarray(load)))
    rc, infos, status, outs = _solve_batch(ctx, kind, probs, bie.make_opts(precision=bie.MIXED_FF), device=True)
    assert rc == bie.OK and set(status) == {bie.OK}
    assert max(i["rel_residual"] for i in infos) <= 1e-12
    for i in range(0, 700, 35):
        g, load = probs[i]
        assert rel2(outs[i], _oracle(kind, g, load)) <= TOL_SOLVE


# ---------------------------------------------------------------------------
# one persistent launch for batches of small problems (one CTA per problem)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [0, 1])
def test_one_launch_small_batches(ctx, kind):
    probs = []
    rng = np.random.default_rng(130 + kind)
    for _ in range(24):  # 1-4 bodies of 40-200 nodes: at most 800 nodes a problem
        g = synth.random_request(rng, max_bodies=4, nodes=(40, 64, 137, 200))
        N = g["body_start"].size - 1
        load = synth.charges(N, rng) if kind == 0 else synth.forces_torques(N, rng).reshape(-1)
        probs.append((g, np.ascontiguousarray(load)))
    g, load = probs[5]
    probs[5] = (g, np.zeros_like(load))  # a zero load: exactly zero out
    opts = bie.make_opts(precision=bie.MIXED_FF)
    rc, infos, status, outs = _solve_batch(ctx, kind, probs, opts, device=True)
    assert rc == bie.OK, (rc, ctx.last_error())
    assert np.all(outs[5] == 0.0)
    for i, ((gg, ld), out) in enumerate(zip(probs, outs)):
        if not np.any(ld):  # problem 5, and one-body problems (mean-free charges are zero)
            assert np.all(out == 0.0)
            continue
        assert rel2(out, _oracle(kind, gg, ld)) <= TOL_SOLVE
        assert infos[i]["rel_residual"] <= 1e-12 and infos[i]["refinements"] >= 1
    # each problem stops on its own: the counts differ between problems
    assert len({q["iters"] for q in infos}) > 1
    # the multi-launch path gives the same solutions
    bie.small_batch_path(False)
    try:
        rc2, _, _, outs2 = _solve_batch(ctx, kind, probs, opts, device=True)
    finally:
        bie.small_batch_path(True)
    assert rc2 == bie.OK
    for (gg, ld), o1, o2 in zip(probs, outs, outs2):
        if np.any(ld):
            assert rel2(o1, o2) <= TOL_SOLVE


def test_one_launch_is_deterministic_and_handles_a_batch_of_one(ctx):
    g = synth.four_discs(seed=3)
    rng = np.random.default_rng(7)
    probs = [(g, synth.charges(4, rng))]
    opts = bie.make_opts(precision=bie.MIXED_FF)
    r1 = _solve_batch(ctx, 0, probs, opts)[3][0]
    r2 = _solve_batch(ctx, 0, probs, opts)[3][0]
    assert np.array_equal(r1, r2)
    assert rel2(r1, _oracle(0, *probs[0])) <= TOL_SOLVE
