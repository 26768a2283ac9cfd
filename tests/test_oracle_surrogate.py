"""Pins of the FP64 surrogate reference (oracle/surrogate_ref.py) against what
mathematics and independent routines fix: finite differences, numpy.correlate,
plain shifts, torch's bfloat16 conversion, the erf form of GELU and the closed
form of one Adam step."""
import math

import numpy as np
import pytest

from oracle import surrogate_ref as S


def small_params(C=6, k=5, dil=(1, 3, 2), seed=1, patch=1):
    p = S.init_params(C=C, k=k, dil=dil, seed=seed)
    rng = np.random.default_rng(seed + 10)
    # patches of `patch` nodes: 4 patch features in, 3 patch outputs
    p.Wl = rng.normal(0, 0.5, (C, 4 * patch))
    # nonzero biases and a larger body so that every term matters
    p.W = [w * 8 for w in p.W]
    p.b = [rng.normal(0, 0.3, C) for _ in dil]
    p.bl = rng.normal(0, 0.3, C)
    p.bp = rng.normal(0, 0.3, 3 * patch)
    p.Wp = rng.normal(0, 0.5, (3 * patch, C))
    return p


def loss_of(p, a, target):
    out, _ = S.forward(p, a, emulate_bf16=False)
    return S.mse(out, target)[0]


@pytest.mark.parametrize("patch", [1, 2])
def test_gradient_matches_central_differences(patch):
    """Every parameter block, exact arithmetic: analytic = (L(p+h) - L(p-h)) / 2h."""
    rng = np.random.default_rng(0)
    p = small_params(patch=patch)
    B, L = 2, 23          # ragged: the dilated taps reach past both ends
    a = rng.normal(0, 1, (B, L, 4 * patch))
    target = rng.normal(0, 1, (B, L, 3 * patch))
    out, cache = S.forward(p, a, emulate_bf16=False)
    _, gout = S.mse(out, target)
    grads = S.backward(p, cache, gout, emulate_bf16=False)
    arrays = p.arrays()
    h = 1e-6
    for arr, g in zip(arrays, grads):
        flat = arr.reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for j in idx:
            old = flat[j]
            flat[j] = old + h
            lp = loss_of(p, a, target)
            flat[j] = old - h
            lm = loss_of(p, a, target)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g.reshape(-1)[j]) <= 1e-6 * max(1.0, abs(fd)), (arr.shape, j, fd,
                                                                              g.reshape(-1)[j])


def test_input_gradient_matches_central_differences():
    """The adjoint of the whole network in its input features."""
    rng = np.random.default_rng(3)
    p = small_params(seed=4)
    a = rng.normal(0, 1, (1, 17, 4))
    target = rng.normal(0, 1, (1, 17, 3))
    out, cache = S.forward(p, a, emulate_bf16=False)
    _, gout = S.mse(out, target)
    S.backward(p, cache, gout, emulate_bf16=False)
    # input gradient = gWl back through the lift: ga = gx0 Wl
    xs = cache["xs"]
    gx = gout @ p.Wp
    for i in reversed(range(len(p.dil))):
        gz = gx * S.gelu_grad(cache["zs"][i])
        gx = gx + S.conv1d_input_grad(gz, cache["W"][i], p.dil[i])
    ga = gx @ p.Wl
    h = 1e-6
    for (l, c) in [(0, 0), (5, 1), (16, 3), (8, 2)]:
        ap, am = a.copy(), a.copy()
        ap[0, l, c] += h
        am[0, l, c] -= h
        fd = (S.mse(S.forward(p, ap, False)[0], target)[0] -
              S.mse(S.forward(p, am, False)[0], target)[0]) / (2 * h)
        assert abs(fd - ga[0, l, c]) <= 1e-6 * max(1.0, abs(fd))
    assert len(xs) == len(p.dil) + 1


@pytest.mark.parametrize("d", [1, 2, 5])
def test_conv_matches_numpy_correlate(d):
    """One input and one output channel: conv1d is numpy's 'same' correlation
    with the dilated kernel."""
    rng = np.random.default_rng(d)
    k, L = 5, 40
    x = rng.normal(0, 1, L)
    w = rng.normal(0, 1, k)
    wd = np.zeros((k - 1) * d + 1)
    wd[::d] = w
    ref = np.correlate(np.pad(x, ((k // 2) * d,)), wd, mode="valid")
    got = S.conv1d(x[None, :, None], w[:, None, None], d)[0, :, 0]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_one_hot_kernel_is_a_shift_and_adjoint_is_transpose():
    rng = np.random.default_rng(7)
    B, L, C, k, d = 2, 19, 3, 5, 3
    x = rng.normal(0, 1, (B, L, C))
    for t in range(k):
        W = np.zeros((k, C, C))
        W[t] = np.eye(C)
        s = (t - k // 2) * d
        ref = np.zeros_like(x)
        for l in range(L):
            if 0 <= l + s < L:
                ref[:, l] = x[:, l + s]
        np.testing.assert_array_equal(S.conv1d(x, W, d), ref)
    # <conv(x), g> = <x, conv^T(g)> and = <W, wgrad(g, x)>
    W = rng.normal(0, 1, (k, 4, C))
    g = rng.normal(0, 1, (B, L, 4))
    lhs = np.sum(S.conv1d(x, W, d) * g)
    assert abs(lhs - np.sum(x * S.conv1d_input_grad(g, W, d))) < 1e-10
    assert abs(lhs - np.sum(W * S.conv1d_weight_grad(g, x, k, d))) < 1e-10


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    v = np.concatenate([rng.normal(0, 1, 5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, 65504.0]])
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16_round(v), ref)
    assert S.bf16_round(1 + 2 ** -8) == 1.0               # tie, to even
    assert S.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6   # tie, to even (up)


def test_gelu_against_erf_form():
    x = np.linspace(-8, 8, 4001)
    exact = 0.5 * x * (1 + np.array([math.erf(v / math.sqrt(2)) for v in x]))
    assert np.max(np.abs(S.gelu(x) - exact)) < 1e-3
    assert S.gelu(0.0) == 0.0 and abs(S.gelu_grad(0.0) - 0.5) < 1e-15
    h = 1e-6
    fd = (S.gelu(x + h) - S.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(S.gelu_grad(x), fd, atol=1e-8)


def test_adam_first_step_closed_form():
    """t = 1: m_hat = g and v_hat = g^2, so the step is lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p0 = np.array([1.0, 2.0, 3.0, 4.0])
    p1, m, v = S.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_conservation_residual_and_l1_error():
    rng = np.random.default_rng(2)
    rho = 1 + 0.1 * rng.random((3, 50))
    u = 0.1 * rng.normal(size=(3, 50))
    T = 1 + 0.1 * rng.random((3, 50))
    n = np.array([0, 2, 4])
    # a permutation of the nodes conserves every total
    perm = rng.permutation(50)
    assert np.all(S.conservation_residual(rho, u, T, rho[:, perm], u[:, perm], T[:, perm], n)
                  < 1e-14)
    # doubling rho changes the mass by 100 %
    assert np.allclose(S.conservation_residual(rho, u, T, 2 * rho, u, T, n), 1.0)
    e = S.l1_error(rho * 1.01, u, T, rho, u, T, [1.4, 1.4, 1.4])
    np.testing.assert_allclose(e, 0.01, rtol=1e-12)
