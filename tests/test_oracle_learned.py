"""Pins of the oracle's learned-guess MLP: analytic backward against central
differences of the FP64 forward, Adam against its closed form, BF16 rounding
against the format definition, and features against their definition."""
import numpy as np
import pytest

import workloads as w
from oracle import learned as ol


def test_bf16_rounding_is_nearest_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert ol.bf16(np.array([1 + 2 ** -8]))[0] == 1.0
    assert ol.bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6
    x = np.linspace(-3, 3, 101)
    r = ol.bf16(x)
    assert np.all(np.abs(r - x) <= 2 ** -8 * np.abs(x) + 1e-30)
    # representable values are fixed points
    assert np.all(ol.bf16(r) == r)


def test_backward_matches_central_differences():
    ol.BF16_ROUNDING = False
    try:
        rng = np.random.default_rng(0)
        params = w.mlp_params(12, 7, 5, seed=1)
        mlp = ol.MLP(params)
        x = rng.standard_normal((9, 12))
        T = rng.standard_normal((9, 5))
        L, grads = mlp.loss_and_grads(x, T)
        for i in range(6):
            p0 = mlp.p[i].copy()
            fd = np.zeros_like(p0)
            it = np.nditer(p0, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                h = 1e-6
                mlp.p[i] = p0.copy(); mlp.p[i][idx] += h
                Lp = mlp.loss_and_grads(x, T)[0]
                mlp.p[i] = p0.copy(); mlp.p[i][idx] -= h
                Lm = mlp.loss_and_grads(x, T)[0]
                fd[idx] = (Lp - Lm) / (2 * h)
            mlp.p[i] = p0
            assert np.allclose(grads[i], fd, rtol=1e-5, atol=1e-9), i
    finally:
        ol.BF16_ROUNDING = True


def test_adam_first_steps_closed_form():
    """With a constant gradient g, Adam's bias-corrected step is lr*sign(g)
    (up to eps) at every step."""
    mlp = ol.MLP([np.zeros((2, 2)), np.zeros(2), np.zeros((2, 2)), np.zeros(2),
                  np.zeros((2, 2)), np.zeros(2)])
    g = [np.full((2, 2), 0.3), np.full(2, -2.0), np.full((2, 2), 1e-3), np.zeros(2),
         np.full((2, 2), 5.0), np.full(2, -1e-2)]
    for k in range(1, 4):
        mlp.adam(g, lr=1e-2)
        for gi, p in zip(g, mlp.p):
            expect = -k * 1e-2 * np.sign(gi) * np.abs(gi) / (np.abs(gi) + 1e-8)
            assert np.allclose(p, np.asarray(expect, np.float32), rtol=1e-5, atol=1e-9)


def test_features_definition():
    rng = np.random.default_rng(2)
    E, nv, nm = 4, 3, 2
    u = [rng.standard_normal((E, nv, nm)) for _ in range(3)]
    x = ol.features(u[:2], u[2], nv)
    assert x.shape == (E, 3 * nv * nm)
    blocks = [u[0], u[0] - u[1], u[2]]
    for k, F in enumerate(blocks):
        xk = x[:, k * nv * nm:(k + 1) * nv * nm].reshape(E, nv, nm)
        # each variable of each block has unit RMS over the mesh
        assert np.allclose(np.sqrt(np.mean(xk ** 2, axis=(0, 2))), 1.0)
        assert np.allclose(xk * np.sqrt(np.mean(F ** 2, axis=(0, 2)))[None, :, None], F)
