"""GPU parity of rh_forward / rh_adjoint (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import oracle
from gpu_common import TOL, rel_l2, rel_max, to_dev, to_np

pytestmark = pytest.mark.gpu

GEOMS = [
    # (n, N, M, h, ds, angles)
    (8, 12, 13, 1.0, 1.0, "uniform"),
    (37, 50, 53, 1.0, 1.0, "uniform"),          # ragged tiles, odd n
    (64, 90, 95, 1.0, 1.0, "uniform"),          # the 64x64 configuration's geometry
    (100, 33, 142, 1.0, 1.0, "random"),         # angles anywhere in [0, 2 pi)
    (48, 40, 70, 0.8, 1.0, "uniform"),          # ds/h = 1.25
    (48, 40, 90, 0.6, 1.0, "uniform"),          # ds/h = 1.67 (3 pixels per interval)
    (40, 30, 45, 1.3, 1.0, "uniform"),          # h > ds
    (33, 17, 1, 1.0, 1.0, "uniform"),           # single bin
    (1, 5, 3, 1.0, 1.0, "uniform"),             # single pixel
    (130, 7, 60, 1.0, 1.0, "uniform"),          # detector narrower than the image
    (60, 24, 90, 0.9, 1.0, "uniform"),          # two pixels per interval, four per interval pair
    (70, 36, 100, 0.95, 1.0, "random"),         # at most three pixels per interval pair
    (200, 45, 283, 1.0, 1.0, "uniform"),        # several 63-bin chunks with a ragged tail
]


def _angles(N, kind, seed=0):
    if kind == "uniform":
        return np.arange(N) * (np.pi / N)
    return np.random.default_rng(seed).uniform(-np.pi, 2 * np.pi, N)


@pytest.fixture(scope="module")
def ct():
    from paper_1810_03275_gb300 import ctrecon
    return ctrecon


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("geom", GEOMS)
def test_forward_adjoint_match_oracle(ct, geom, dtype):
    n, N, M, h, ds, kind = geom
    th = _angles(N, kind, n)
    plan = ct.Plan(n, N, M, angles=th, h=h, ds=ds, dtype=dtype)
    geo = oracle.Geometry(n, N, M, h=h, ds=ds, theta=th)
    rng = np.random.default_rng(n + N)
    u = rng.standard_normal((n, n))
    g = rng.standard_normal((N, M))
    ref_f = oracle.rh_forward(u, geo)
    ref_b = oracle.rh_adjoint(g, geo)
    got_f = to_np(plan.rh_forward(to_dev(u, plan.torch_dtype)))
    got_b = to_np(plan.rh_adjoint(to_dev(g, plan.torch_dtype)))
    tol = TOL[dtype]
    assert rel_l2(got_f, ref_f) < tol, rel_l2(got_f, ref_f)
    assert rel_l2(got_b, ref_b) < tol, rel_l2(got_b, ref_b)
    assert rel_max(got_f, ref_f) < 10 * tol
    assert rel_max(got_b, ref_b) < 10 * tol


def test_symmetric_path_selection(ct):
    """FP32 and BF16 plans with uniform angles over [0, pi) take the symmetric path: an even
    count in jobs of up to four angles, an odd count in (N + 1) / 2 pair jobs (theta with
    pi - theta); angles outside [0, pi), FP64 plans and pixels smaller than ds/2 (three per
    interval) project angle by angle."""
    uni = lambda N: np.arange(N) * (np.pi / N)
    p = ct.Plan(64, 90, 95, angles=uni(90))
    assert 0 < p.symmetric_jobs <= 45
    assert ct.Plan(512, 720, 729, angles=uni(720)).symmetric_jobs == 181
    assert ct.Plan(64, 45, 95, angles=uni(45)).symmetric_jobs == 23
    assert ct.Plan(64, 33, 95, angles=_angles(33, "random", 1)).symmetric_jobs == 0
    assert ct.Plan(64, 90, 95, angles=uni(90), dtype="f64").symmetric_jobs == 0
    assert ct.Plan(64, 90, 95, angles=uni(90), dtype="bf16").symmetric_jobs > 0
    assert ct.Plan(48, 40, 70, angles=uni(40), h=0.8).symmetric_jobs > 0      # two pixels per interval
    assert ct.Plan(48, 40, 70, angles=uni(40), h=0.6).symmetric_jobs == 0     # three pixels per interval


@pytest.mark.parametrize("case", ["duplicated", "shuffled", "partial"])
def test_symmetric_path_angle_sets(ct, case):
    """The symmetric path on angle sets that fill its jobs unevenly: every angle twice,
    a shuffled uniform set, and a set where most jobs miss channels."""
    n, M = 70, 101
    base = np.arange(36) * (np.pi / 36)
    if case == "duplicated":
        th = np.concatenate([base, base])
    elif case == "shuffled":
        th = np.random.default_rng(4).permutation(base)
    else:
        th = base[np.arange(36) % 3 != 1]       # 24 angles, two per job on average
    N = th.shape[0]
    plan = ct.Plan(n, N, M, angles=th)
    assert plan.symmetric_jobs > 0
    geo = oracle.Geometry(n, N, M, theta=th)
    rng = np.random.default_rng(N)
    u = rng.standard_normal((n, n))
    g = rng.standard_normal((N, M))
    got_f = to_np(plan.rh_forward(to_dev(u, plan.torch_dtype)))
    got_b = to_np(plan.rh_adjoint(to_dev(g, plan.torch_dtype)))
    assert rel_l2(got_f, oracle.rh_forward(u, geo)) < TOL["f32"]
    assert rel_l2(got_b, oracle.rh_adjoint(g, geo)) < TOL["f32"]


@pytest.mark.parametrize("geom", [(64, 90, 95), (96, 60, 137)])
def test_backprojection_group_splits_agree(ct, geom):
    """Every group split the plan allows (symmetric path: jobs, per-angle path: angles)
    gives the same R_h^* up to FP32 summation order, and the oracle's."""
    n, N, M = geom
    th = np.arange(N) * (np.pi / N)
    geo = oracle.Geometry(n, N, M, theta=th)
    g = np.random.default_rng(N).standard_normal((N, M))
    ref = oracle.rh_adjoint(g, geo)
    for th_set in (th, th[:-1]):                           # even count: symmetric; odd: per angle
        plan = ct.Plan(n, th_set.shape[0], M, angles=th_set)
        gg = to_dev(g[:th_set.shape[0]], plan.torch_dtype)
        r = ref if th_set is th else oracle.rh_adjoint(g[:-1], oracle.Geometry(n, N - 1, M, theta=th_set))
        got = {}
        for G in range(1, 9):
            try:
                plan.set_bp_groups(G)
            except Exception:
                continue
            assert plan.bp_groups == G
            got[G] = to_np(plan.rh_adjoint(gg))
            assert rel_l2(got[G], r) < TOL["f32"], G
        assert len(got) >= 2
        first = next(iter(got.values()))
        for v in got.values():
            assert rel_l2(v, first) < 1e-6


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_adjoint_identity_on_gpu(ct, dtype):
    """<R u, g> = <u, R^* g> for the GPU pair (exact transpose: same integer weights)."""
    import torch
    n, N, M = 96, 120, 137
    plan = ct.Plan(n, N, M, dtype=dtype)
    gen = torch.Generator(device="cuda").manual_seed(3)
    u = torch.randn((n, n), generator=gen, device="cuda", dtype=plan.torch_dtype)
    g = torch.randn((N, M), generator=gen, device="cuda", dtype=plan.torch_dtype)
    lhs = float((plan.rh_forward(u).double() * g.double()).sum())
    rhs = float((u.double() * plan.rh_adjoint(g).double()).sum())
    scale = float(u.double().norm() * g.double().norm())
    assert abs(lhs - rhs) / scale < (1e-6 if dtype == "f32" else 1e-13)


def test_full_size_sampled_entries(ct):
    """512 x 512, 720 angles, 729 bins (the benchmark geometry) in the benchmark's
    launch configuration: 300 sampled bins and pixels against brute-force oracle
    entries (hat weights, one output at a time)."""
    n, N, M = 512, 720, 729
    th = np.arange(N) * (np.pi / N)
    plan = ct.Plan(n, N, M, angles=th)
    geo = oracle.Geometry(n, N, M, theta=th)
    rng = np.random.default_rng(11)
    u = rng.uniform(0, 1, (n, n))
    g = rng.standard_normal((N, M))
    got_f = to_np(plan.rh_forward(to_dev(u, plan.torch_dtype)))
    got_b = to_np(plan.rh_adjoint(to_dev(g, plan.torch_dtype)))
    ls = rng.integers(0, N, 300)
    ks = rng.integers(0, M, 300)
    ref = oracle.rh_forward_entries(u, geo, ls, ks)
    assert rel_max(got_f[ls, ks], ref) < 1e-5
    is_ = rng.integers(0, n, 300)
    js = rng.integers(0, n, 300)
    ref = oracle.rh_adjoint_entries(g, geo, is_, js)
    assert rel_l2(got_b[is_, js], ref) < 1e-5
    # mass per angle equals the image sum (footprint inside the detector)
    np.testing.assert_allclose(got_f.sum(1), u.sum(), rtol=1e-5)


def test_point_projection(ct):
    """Single pixel: each projection carries unit mass centred at x cos + y sin."""
    n, N, M = 16, 9, 31
    plan = ct.Plan(n, N, M)
    u = np.zeros((n, n))
    u[13, 4] = 1.0
    got = to_np(plan.rh_forward(to_dev(u, plan.torch_dtype)))
    th = np.arange(N) * np.pi / N
    pos = (13 - 7.5) * np.cos(th) + (4 - 7.5) * np.sin(th) + 15
    np.testing.assert_allclose(got.sum(1), 1.0, atol=1e-6)
    np.testing.assert_allclose((got * np.arange(M)).sum(1), pos, atol=2e-5)



@pytest.mark.parametrize("geom", [g for g in GEOMS if g[5] == "uniform" and g[0] > 1] +
                         [(512, 720, 729, 1.0, 1.0, "uniform"), (96, 120, 137, 1.0, 1.0, "uniform")])
def test_staged_forward_shape(ct, geom):
    """The staged forward projector (shape (4, 1): four adjacent jobs per CTA share a
    cp.async-staged window of the orbit image) on every symmetric-path geometry, FP32 and
    BF16: equal to the default shape up to FP32 summation order and to the oracle."""
    import torch
    n, N, M, h, ds, _ = geom
    th = np.arange(N) * (np.pi / N)
    for dtype in ("f32", "bf16"):
        plan = ct.Plan(n, N, M, angles=th, h=h, ds=ds, dtype=dtype)
        if plan.symmetric_jobs == 0:
            pytest.skip("per-angle path")
        u = torch.as_tensor(np.random.default_rng(n).standard_normal((n, n)), dtype=torch.float32,
                            device="cuda").to(plan.op_dtype)
        base = to_np(plan.rh_forward(u))
        plan.set_fwd_shape(4, 1)
        got = to_np(plan.rh_forward(u))
        ref = oracle.rh_forward(u.double().cpu().numpy(), oracle.Geometry(n, N, M, h=h, ds=ds, theta=th))
        assert rel_l2(got, base) < 2e-6, dtype
        assert rel_l2(got, ref) < 1e-5, dtype


def test_staged_shape_refused_where_window_exceeds_shared_memory(ct):
    """A plan whose staged window would not fit one CTA's shared memory (2048^2, 4 views)
    is still created, and refuses the staged shape with CTR_EUNSUPPORTED; the default
    shape projects as before."""
    import torch
    n, N, M = 2048, 4, 2897
    plan = ct.Plan(n, N, M, angles=np.arange(N) * (np.pi / N))
    if plan.symmetric_jobs == 0:
        pytest.skip("per-angle path")
    with pytest.raises(ct.CtrError) as e:
        plan.set_fwd_shape(4, 1)
    assert e.value.status == -6      # CTR_EUNSUPPORTED
    u = torch.ones((n, n), device="cuda")
    g = to_np(plan.rh_forward(u))
    assert np.all(np.isfinite(g)) and g.max() > 0


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("n,N,M", [(64, 91, 95), (130, 181, 185), (512, 721, 729)])
def test_odd_view_count_symmetric_path(ct, n, N, M, dtype):
    """Odd view counts take the symmetric path with pair jobs (channels {0, 1} or {2, 3}
    only): both projectors match the oracle, and the operators stay exact transposes."""
    import torch
    th = np.arange(N) * (np.pi / N)
    plan = ct.Plan(n, N, M, angles=th, dtype=dtype)
    assert plan.symmetric_jobs == (N + 1) // 2
    geo = oracle.Geometry(n, N, M, theta=th)
    rng = np.random.default_rng(N)
    u = rng.standard_normal((n, n))
    g = rng.standard_normal((N, M))
    if dtype == "bf16":                       # bfloat16-representable inputs: equal to FP32 up to rounding
        u = torch.as_tensor(u, dtype=torch.float32).to(torch.bfloat16).double().numpy()
        g = torch.as_tensor(g, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    gf = to_np(plan.rh_forward(to_dev(u, torch.float32).to(plan.op_dtype)))
    ub = to_np(plan.rh_adjoint(to_dev(g, torch.float32).to(plan.op_dtype)))
    assert rel_l2(gf, oracle.rh_forward(u, geo)) < 1e-5
    assert rel_l2(ub, oracle.rh_adjoint(g, geo)) < 1e-5
    lhs, rhs = float(np.sum(gf * g)), float(np.sum(u * ub))
    # FP32 rounding of either side is bounded relative to |R u| |g| (Cauchy-Schwarz), not to
    # the inner product itself, which random signs make much smaller
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(gf) * np.linalg.norm(g)


@pytest.mark.parametrize("N", [6, 7])
def test_largest_image(ct, N):
    """4096 x 4096 with 5793 bins (the widest detector of the plans here), a few views (even:
    symmetric path, odd: pair jobs): both projectors against the oracle in FP32, and the
    adjoint identity."""
    import torch
    n, M = 4096, 5793
    th = np.arange(N) * (np.pi / N)
    plan = ct.Plan(n, N, M, angles=th)
    geo = oracle.Geometry(n, N, M, theta=th)
    rng = np.random.default_rng(N)
    u = rng.standard_normal((n, n))
    g = rng.standard_normal((N, M))
    gf = to_np(plan.rh_forward(to_dev(u, torch.float32)))
    ub = to_np(plan.rh_adjoint(to_dev(g, torch.float32)))
    assert rel_l2(gf, oracle.rh_forward(u, geo)) < 1e-5
    assert rel_l2(ub, oracle.rh_adjoint(g, geo)) < 1e-5
    lhs, rhs = float(np.sum(gf * g)), float(np.sum(u * ub))
    # FP32 rounding of either side is bounded relative to |R u| |g| (Cauchy-Schwarz), not to
    # the inner product itself, which random signs make much smaller
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(gf) * np.linalg.norm(g)
