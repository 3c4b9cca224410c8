"""Pins of the FP64 reference of the warm-start network (oracle/mlp.py): the
gradient against central finite differences of the loss, a closed form for
the zero network, and the bfloat16 rounding rule."""
import numpy as np

from oracle import mlp

NIN = mlp.DIMS[0][0]


def _net(rng, scale=1.0):
    p = np.zeros(mlp.NPARAM)
    off = 0
    for i, o in mlp.DIMS:
        p[off:off + i * o] = scale * rng.standard_normal(i * o) / np.sqrt(i)
        off += i * o
        p[off:off + o] = 0.1 * rng.standard_normal(o)
        off += o
    return p


def _norm(rng):
    return (rng.standard_normal(NIN), rng.uniform(0.5, 2.0, NIN),
            rng.standard_normal(192), rng.uniform(0.5, 2.0, 192))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _net(rng)
    norm = _norm(rng)
    x = rng.standard_normal((3, NIN))
    t = rng.standard_normal((3, 192))
    _, g = mlp.loss_and_grad(p, x, t, norm, bf16=False)
    # a few entries of every weight and bias block
    idx, off = [], 0
    for i, o in mlp.DIMS:
        idx += list(off + rng.integers(0, i * o, 4))
        off += i * o
        idx += list(off + rng.integers(0, o, 2))
        off += o
    for k in idx:
        h = 1e-5
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss_and_grad(pp, x, t, norm, bf16=False)[0] -
              mlp.loss_and_grad(pm, x, t, norm, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_zero_network_closed_form():
    rng = np.random.default_rng(1)
    norm = _norm(rng)
    x = rng.standard_normal((5, NIN))
    t = rng.standard_normal((5, 192))
    y, _ = mlp.forward(np.zeros(mlp.NPARAM), x, norm)
    np.testing.assert_allclose(y, np.tile(norm[2], (5, 1)), rtol=0, atol=0)
    loss, g = mlp.loss_and_grad(np.zeros(mlp.NPARAM), x, t, norm)
    that = (t - norm[2]) / norm[3]
    assert abs(loss - 0.5 * np.sum(that ** 2) / 5) <= 1e-12 * loss
    # only the output bias has a gradient: -sum(t_hat) / B
    np.testing.assert_allclose(g[-192:], -that.sum(axis=0) / 5, rtol=1e-12, atol=1e-15)
    assert np.all(g[:-192] == 0)


def test_bf16_rounding_ties_to_even():
    one = 1.0
    vals = np.array([one, one + 2.0 ** -8, one + 3 * 2.0 ** -8, one + 2.0 ** -7, -2.5,
                     one + 2.0 ** -8 + 2.0 ** -20])
    exp = np.array([one, one, one + 2.0 ** -6, one + 2.0 ** -7, -2.5, one + 2.0 ** -7])
    np.testing.assert_array_equal(mlp.bf16_round(vals), exp)
    assert mlp.bf16_bits(np.array([1.0]))[0] == 0x3F80


def test_gradient_magnitudes_equal_the_gradient_when_nothing_cancels():
    """With non-negative weights, biases, normalised inputs and output errors
    (targets below the outputs), no term of the backward pass is negative, so
    the magnitude sums are the gradient itself; in general they bound it."""
    rng = np.random.default_rng(4)
    p = np.abs(_net(rng))
    norm = _norm(rng)
    x = norm[0] + norm[1] * np.abs(rng.standard_normal((6, NIN)))
    y, _ = mlp.forward(p, x, norm, bf16=False)
    t = y - np.abs(rng.standard_normal(y.shape)) - 0.1
    _, g = mlp.loss_and_grad(p, x, t, norm, bf16=False)
    m = mlp.grad_magnitudes(p, x, t, norm, bf16=False)
    np.testing.assert_allclose(m, g, rtol=1e-12, atol=1e-300)
    # random signs: |g| <= magnitude sum, entry by entry
    p2, t2 = _net(rng), rng.standard_normal((6, 192))
    x2 = rng.standard_normal((6, NIN))
    _, g2 = mlp.loss_and_grad(p2, x2, t2, norm, bf16=False)
    m2 = mlp.grad_magnitudes(p2, x2, t2, norm, bf16=False)
    assert np.all(np.abs(g2) <= m2 * (1 + 1e-12))
