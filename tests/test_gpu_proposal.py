"""Learned proposal on the GPU: the ranking network's BF16 tensor-core
forward and backward against the CPU reference (oracle/mlp_ref.py, pinned by
finite differences), training on checker labels, and ranked search against
plain enumeration."""
import numpy as np
import pytest

from oracle import mlp_ref as M
from paper_1308_3203_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    return racecheck


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def feature_rows(rc, n, seed):
    """Real candidate features, plus noise rows, n in total."""
    from paper_1308_3203_gb300 import proposal
    rows = []
    s = 0
    while sum(len(r) for r in rows) < n // 2:
        _, items = proposal.kernel_candidates(1000 + seed * 100 + s)
        rows.append(rc.features(items))
        s += 1
    X = np.concatenate(rows)[: n // 2] if rows else np.zeros((0, M.IN), np.float32)
    rng = np.random.default_rng(seed)
    return np.concatenate([X, rng.uniform(0, 1, size=(n - len(X), M.IN)).astype(np.float32)])


def test_params_round_trip(rc):
    m = rc.MLP(seed=3, capacity=256)
    p = m.params()
    assert p.shape == (M.N_PARAMS,) and np.all(p[M.offsets()["b1"][0]:M.offsets()["b1"][1]] == 0)
    q = M.init_params(9).astype(np.float32)
    m.set_params(q)
    np.testing.assert_array_equal(m.params(), q)


@pytest.mark.parametrize("n", [1, 63, 1000, 4097])
def test_forward_matches_reference(rc, n):
    m = rc.MLP(seed=1, capacity=2048)  # n > capacity runs in passes
    p = M.init_params(5).astype(np.float32)
    m.set_params(p)
    X = feature_rows(rc, n, n)
    got = m.forward(cuda(X)).cpu().numpy()
    want, _ = M.forward(p, X, bf16_points=True)
    exact, _ = M.forward(p, X, bf16_points=False, dtype=np.float64)
    # same rounding points: only FP32 summation order differs (it can move a
    # hidden value across a BF16 rounding boundary, one BF16 ulp = 2^-8)
    np.testing.assert_allclose(got, want, atol=4e-3, rtol=0)
    np.testing.assert_allclose(got, exact, atol=3e-2, rtol=0)


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 4097])
def test_tcgen05_forward_matches(rc, n):
    """The tcgen05 forward (TMEM accumulators), its three layers in one
    launch and one launch per layer, against the mma.sync forward and the
    CPU reference on the same parameters and rows (ragged 128-row tiles,
    several passes over the capacity)."""
    m = rc.MLP(seed=1, capacity=2048)
    p = M.init_params(5).astype(np.float32)
    m.set_params(p)
    X = feature_rows(rc, n, 50 + n)
    m.set_backend(0)
    a = m.forward(cuda(X)).cpu().numpy()
    m.set_backend(2)
    c = m.forward(cuda(X)).cpu().numpy()
    m.set_backend(1)
    b = m.forward(cuda(X)).cpu().numpy()
    assert m.backend_error() == 0
    want, _ = M.forward(p, X, bf16_points=True)
    np.testing.assert_allclose(b, a, atol=4e-3, rtol=0)
    np.testing.assert_allclose(b, want, atol=4e-3, rtol=0)
    # the fused layers compute the same FP32 sums of the same BF16 products
    # and round them at the same points: the same bits
    np.testing.assert_array_equal(b, c)


# Element-wise bar of a gradient against the reference with the same BF16
# rounding points: 2^-6 of the largest magnitude in the element's parameter
# block.  The kernels and the reference round at the same points and differ
# in FP32 summation order only; the CPU evaluation of the same rounding
# points in float32 against float64 (uniform features, 7-2500 rows) differs
# by at most 3.5e-3 of the block maximum (the order moving a hidden value
# across a BF16 rounding boundary, one BF16 ulp = 2^-8 relative, which the
# later layers carry), so 2^-6 = 1.6e-2 leaves a margin of 4.5.
GRAD_ATOL_OF_BLOCK_MAX = 2.0 ** -6


def check_gradient(g, want, exact):
    for name, (a, b, _) in M.offsets().items():
        atol = GRAD_ATOL_OF_BLOCK_MAX * max(np.abs(want[a:b]).max(), 1e-30)
        np.testing.assert_allclose(g[a:b], want[a:b], rtol=0, atol=atol, err_msg=name)
        # against the exact float64 network: no farther than the rounding points
        # themselves put the reference, plus the bar above (in the L2 norm)
        gap, ref_gap = np.linalg.norm(g[a:b] - exact[a:b]), np.linalg.norm(want[a:b] - exact[a:b])
        assert gap <= ref_gap + GRAD_ATOL_OF_BLOCK_MAX * np.linalg.norm(exact[a:b]), (name, gap, ref_gap)


@pytest.mark.parametrize("backend", [0, 1])
@pytest.mark.parametrize("n", [7, 777, 2500])
def test_gradient_matches_reference(rc, n, backend):
    """Both backends: mma.sync (0) and tcgen05 (1) for every product; every
    gradient element against the BF16-point reference."""
    m = rc.MLP(seed=2, capacity=4096)
    m.set_backend(backend)
    p = M.init_params(11).astype(np.float32)
    m.set_params(p)
    X = feature_rows(rc, n, 7 + n)
    y = (np.random.default_rng(n).random(n) < 0.3).astype(np.float32)
    g, loss = m.grad(cuda(X), cuda(y))
    want_loss, want = M.loss_and_grad(p, X, y, bf16_points=True)
    _, exact = M.loss_and_grad(p, X, y, bf16_points=False, dtype=np.float64)
    assert loss == pytest.approx(want_loss, rel=2e-3)
    check_gradient(g, want, exact)
    # the parameters did not move
    np.testing.assert_array_equal(m.params(), p)
    assert m.backend_error() == 0


@pytest.mark.parametrize("backend", [0, 1, 2])
def test_adam_steps_match_reference(rc, backend):
    """Three training steps (one minibatch of all rows per call, rows in the
    library's shuffled order) against the float64 Adam update of
    oracle/mlp_ref.py applied to the gradient the GPU computes at each step
    (rc_mlp_grad on the same rows in the same order, before the step):
    parameters and moments carried from step to step.  The update is FP32 on
    the GPU; the bar is one part in 10^5 of the learning rate per element on
    top of 10^-6 relative to the parameter."""
    n, lr = 600, 2e-3
    m = rc.MLP(seed=4, capacity=1024)
    m.set_backend(backend)
    p = M.init_params(21).astype(np.float32)
    m.set_params(p)
    X = feature_rows(rc, n, 99)
    y = (np.random.default_rng(5).random(n) < 0.3).astype(np.float32)
    mom, vel = np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    cur = p.astype(np.float64)
    for t in (1, 2, 3):
        seed = 100 + t
        perm, _ = M.shuffle(n, seed)
        g, _ = m.grad(cuda(X[perm]), cuda(y[perm]))
        _, want_g = M.loss_and_grad(cur.astype(np.float32), X[perm], y[perm], bf16_points=True)
        _, exact_g = M.loss_and_grad(cur, X[perm], y[perm], bf16_points=False, dtype=np.float64)
        check_gradient(g, want_g, exact_g)
        m.train(cuda(X), cuda(y), epochs=1, batch=n, lr=lr, seed=seed)
        cur, mom, vel = M.adam_step(cur, g.astype(np.float64), mom, vel, t, lr)
        got = m.params().astype(np.float64)
        np.testing.assert_allclose(got, cur, rtol=1e-6, atol=1e-5 * lr, err_msg=f"step {t}")
        cur = got  # carry the GPU's FP32 parameters (its rounding) into the next step
    assert m.backend_error() == 0


def test_training_ranks_racy_candidates_first(rc):
    """Train on checker labels of 240 kernels' candidates; on 60 held-out
    kernels the ranked search reaches a racy candidate in fewer checks and
    less time than enumeration, every reported race is the checker's, and
    the ranking finds a race on most racy kernels within 2 checks."""
    from paper_1308_3203_gb300 import proposal
    X, y, _ = proposal.dataset(range(240))
    assert 0.05 < y.mean() < 0.6
    m = rc.MLP(seed=0, capacity=4096)
    losses = m.train(cuda(X), cuda(y), epochs=12, batch=1024, lr=2e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0], losses
    res = proposal.compare_search(m, range(100000, 100060))
    assert res["racy_kernels"] >= 20
    rk = res["ranked"]
    assert rk["checks_mean"] < res["enum_checks_mean"]
    assert rk["check_speedup"] > 1.5, res
    assert rk["recall"] == 1.0 and rk["recall_at_2"] >= 0.7, res
    for r in res["rows"]:
        for k in ("ranked", "overlap", "rule", "rule_overlap"):
            assert r[f"{k}_found"] == r["racy"]  # every search sees every candidate when needed


def test_search_ranked_orders_as_rc_search_with_the_same_scores(rc):
    """rc_search_ranked (features, scores and checks in one call) meets the
    same first racy candidate after the same checks as rc_search given the
    scores computed step by step: the network's (an untrained one will do)
    and the rule's."""
    from paper_1308_3203_gb300 import proposal
    m = rc.MLP(seed=3, capacity=256)
    for s in range(200000, 200012):
        _, items = proposal.kernel_candidates(s)
        X = rc.features(items)
        for model, sc in ((m, proposal.scores(m, X)), (None, proposal.rule_scores(X))):
            want = rc.search(items, scores=sc)
            got = rc.search_ranked(items, model)
            assert (got["first"], got["checks"]) == (want["first"], want["checks"]), (s, model)
            assert got["checks_unranked"] == 0
            if got["first"] >= 0:
                assert got["report"]["status"] == rc.RACY
            for lim in (1, 3):
                g2 = rc.search_ranked(items, model, max_checks=lim)
                w2 = rc.search(items, scores=sc, max_checks=lim)
                assert (g2["first"], g2["checks"]) == (w2["first"], w2["checks"])


def test_search_ranked_overlap_finds_what_enumeration_finds(rc):
    """With RC_RANK_OVERLAP every race still comes from a check (the report
    is racy), the search finds one exactly when enumeration does, and no
    candidate is checked twice (checks <= candidates)."""
    from paper_1308_3203_gb300 import proposal
    m = rc.MLP(seed=4, capacity=256)
    for s in range(200100, 200116):
        _, items = proposal.kernel_candidates(s)
        enum = rc.search(items)
        for model in (m, None):
            got = rc.search_ranked(items, model, overlap=True)
            assert (got["first"] >= 0) == (enum["first"] >= 0), s
            assert got["checks_unranked"] <= got["checks"] <= len(items)
            if got["first"] >= 0:
                assert got["report"]["status"] == rc.RACY
                one = rc.check(items[got["first"]][0], items[got["first"]][1], items[got["first"]][2],
                               items[got["first"]][3])
                assert one["status"] == rc.RACY
