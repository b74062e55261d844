"""Pins of the CPU reference of the ranking network (no GPU): its gradient
against central finite differences of its own loss in float64, its bfloat16
rounding against torch's conversion, and closed forms of a degenerate
network."""
import numpy as np
import pytest

from oracle import mlp_ref as M


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=4000).astype(np.float32) * 10.0 ** rng.integers(-8, 8, size=4000),
                        # exact ties between two bfloat16 values: low 16 bits 0x8000
                        (np.arange(1, 2001, dtype=np.uint32) << 16 | 0x8000).view(np.float32),
                        np.array([0.0, -0.0, 1.0, -1.0, 3.0e38], dtype=np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(M.bf16(x), want)


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    X = rng.normal(size=(6, M.IN))
    y = rng.integers(0, 2, size=6).astype(np.float64)
    _, g = M.loss_and_grad(p, X, y, bf16_points=False, dtype=np.float64)
    off = M.offsets()
    idx = []
    for name, (a, b, _) in off.items():  # parameters of every block
        idx += list(rng.choice(np.arange(a, b), size=min(12, b - a), replace=False))
    eps = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += eps
        lp, _ = M.loss_and_grad(q, X, y, bf16_points=False, dtype=np.float64)
        q[i] -= 2 * eps
        lm, _ = M.loss_and_grad(q, X, y, bf16_points=False, dtype=np.float64)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_zero_network_closed_form():
    """All weights and hidden biases zero, b4 = c: every score is
    sigmoid(c), the loss is mean(log(1 + e^c) - y c), dL/db4 = mean(p - y)
    and every other gradient is zero (the hidden units are all 0)."""
    c = 0.7
    p = np.zeros(M.N_PARAMS)
    p[-1] = c
    X = np.random.default_rng(1).normal(size=(5, M.IN))
    y = np.array([1, 0, 1, 1, 0], dtype=np.float64)
    prob, _ = M.forward(p, X, bf16_points=False, dtype=np.float64)
    s = 1 / (1 + np.exp(-c))
    np.testing.assert_allclose(prob, s, rtol=1e-15)
    loss, g = M.loss_and_grad(p, X, y, bf16_points=False, dtype=np.float64)
    assert loss == pytest.approx(np.mean(np.log1p(np.exp(c)) - y * c), rel=1e-14)
    assert g[-1] == pytest.approx(np.mean(s - y), rel=1e-13)
    assert np.all(g[:-1] == 0)


def test_one_unit_path_closed_form():
    """Only unit 0 of each layer is live: W1[0] = e_0, W2[0][0] = W3[0][0] = 1,
    w4[0] = 1.  For x_0 > 0 the score is sigmoid(x_0 + b4) and
    dL/dW1[0][0] = (p - y) x_0 / n, for x_0 < 0 it is sigmoid(b4) with a
    zero W1 gradient (the ReLU is closed)."""
    d = {k: np.zeros(s) for k, s in M.SIZES}
    d["W1"][0, 0] = 1
    d["W2"][0, 0] = 1
    d["W3"][0, 0] = 1
    d["w4"][0] = 1
    d["b4"][0] = -0.25
    p = M.pack(d)
    X = np.zeros((2, M.IN))
    X[0, 0], X[1, 0] = 1.5, -2.0
    y = np.array([0.0, 1.0])
    prob, _ = M.forward(p, X, bf16_points=False, dtype=np.float64)
    np.testing.assert_allclose(prob, 1 / (1 + np.exp(-np.array([1.25, -0.25]))), rtol=1e-14)
    _, g = M.loss_and_grad(p, X, y, bf16_points=False, dtype=np.float64)
    G = M.unpack(g)
    assert G["W1"][0, 0] == pytest.approx((prob[0] - 0.0) * 1.5 / 2, rel=1e-13)
    assert G["b4"][0] == pytest.approx(((prob[0] - 0) + (prob[1] - 1)) / 2, rel=1e-13)


def test_bf16_points_stay_close_to_exact():
    """Rounding at the BF16 points changes scores by far less than they vary."""
    p = M.init_params(4)
    X = np.random.default_rng(4).normal(size=(64, M.IN))
    a, _ = M.forward(p, X, bf16_points=True)
    b, _ = M.forward(p, X, bf16_points=False, dtype=np.float64)
    assert np.max(np.abs(a - b)) < 0.02


def test_bf16_rounding_points_on_one_path():
    """The one-unit path with hidden biases 2^-9 and x_0 = 1 + 2^-8.  At the
    BF16 points the input, the weights and every hidden activation are
    rounded to bfloat16 (biases stay float32; the bfloat16 spacing at 1 is
    2^-7): x_0 is a tie between 1 and 1 + 2^-7 and goes to the even 1, and
    each hidden value 1 + 2^-9 rounds back to 1, so the score is
    sigmoid(1 + b4).  Without rounding it is sigmoid(1 + 2^-8 + 3 * 2^-9 + b4)."""
    d = {k: np.zeros(s) for k, s in M.SIZES}
    d["W1"][0, 0] = d["W2"][0, 0] = d["W3"][0, 0] = d["w4"][0] = 1
    d["b1"][0] = d["b2"][0] = d["b3"][0] = 2.0 ** -9
    d["b4"][0] = -0.25
    p = M.pack(d)
    X = np.zeros((1, M.IN))
    X[0, 0] = 1 + 2.0 ** -8
    a, _ = M.forward(p, X, bf16_points=True)
    assert a[0] == pytest.approx(1 / (1 + np.exp(-0.75)), rel=1e-6)
    b, _ = M.forward(p, X, bf16_points=False, dtype=np.float64)
    assert b[0] == pytest.approx(1 / (1 + np.exp(-(0.75 + 2.0 ** -8 + 3 * 2.0 ** -9))), rel=1e-14)


# ---- the optimiser's update (Adam, Kingma & Ba, Algorithm 1)

LR, EPS = 1e-3, 1e-8


def test_adam_first_step_closed_form():
    """With zero moments and t = 1 the corrected moments are g and g^2
    exactly, so every parameter moves by lr * g / (|g| + eps): lr times its
    gradient's sign wherever |g| >> eps, nothing where g = 0."""
    rng = np.random.default_rng(0)
    p = rng.normal(size=1000)
    g = rng.normal(size=1000) * 10.0 ** rng.integers(-9, 2, size=1000)
    g[:10] = 0
    z = np.zeros(1000)
    p1, m1, v1 = M.adam_step(p, g, z, z, 1, LR)
    np.testing.assert_allclose(p1, p - LR * g / (np.abs(g) + EPS), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(p1[:10], p[:10])
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_adam_constant_gradient_moves_by_lr_every_step():
    """A gradient held constant: the first moment after t steps is
    (1 - 0.9^t) g and the second (1 - 0.999^t) g^2, which the bias
    corrections divide back to g and g^2, so steps 1..6 each move by
    lr * g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 2e-4, -7e-6])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 7):
        q, m, v = M.adam_step(p, g, m, v, t, LR)
        np.testing.assert_allclose(q - p, -LR * g / (np.abs(g) + EPS), rtol=1e-9)
        p = q


def test_adam_alternating_gradient_closed_form():
    """Gradients g then -g: after two steps the first moment is
    0.9 * 0.1 g - 0.1 g = -0.01 g, corrected by 1 - 0.81 to -g / 19; the
    second is (1 - 0.999^2) g^2, corrected to g^2 exactly.  So the second
    step moves by +lr * (g / 19) / (|g| + eps)."""
    g = np.array([1.0, -4.0, 0.25])
    z = np.zeros(3)
    p1, m, v = M.adam_step(z, g, z, z, 1, LR)
    p2, m, v = M.adam_step(p1, -g, m, v, 2, LR)
    np.testing.assert_allclose(m, -0.01 * g, rtol=1e-12)
    np.testing.assert_allclose(p2 - p1, LR * (g / 19) / (np.abs(g) + EPS), rtol=1e-12)


def test_shuffle_is_fisher_yates_over_splitmix64():
    """The row order of a training epoch: a permutation, drawn from
    splitmix64, whose first outputs from state 0 are the published
    0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f (for n = 4
    the swaps take those outputs mod 4, 3 and 2)."""
    perm, state = M.shuffle(4, 0)
    a = list(range(4))
    for i, r in zip((3, 2, 1), (0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f)):
        j = r % (i + 1)
        a[i], a[j] = a[j], a[i]
    assert perm.tolist() == a
    assert state == 3 * 0x9E3779B97F4A7C15 % (1 << 64)
    for n, seed in ((1, 5), (1000, 7), (4097, 1 << 63)):
        perm, _ = M.shuffle(n, seed)
        assert sorted(perm.tolist()) == list(range(n))
