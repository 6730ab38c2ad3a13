"""Pins of the oracle's Adam update (oracle/nn.py: adam_update), the optimiser
of the force-matching training (the paper names none; Adam with
b1 = 0.9, b2 = 0.999, eps = 1e-8 is the reading used):

- two steps on one weight against values worked by hand
  (tests/golden/adam_two_steps.json, Kingma and Ba 2015, Algorithm 1);
- the closed forms of a constant gradient: the bias-corrected moments are g
  and g^2 at every step, so each step moves a weight by lr g / (|g| + eps);
- the first step moves every trainable weight by lr |g| / (|g| + eps)
  whatever the gradient's scale;
- the feature normalisation (mu, inv_sd) and the energy scale and shift are
  not trained: those entries never move."""
import json
import os

import numpy as np
import pytest

from oracle import nn

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "adam_two_steps.json")))
WIDTH, DEPTH = 8, 2
NP = nn.n_params(WIDTH, DEPTH)
TRAINABLE = slice(2 * nn.N_IN, NP - 2)


def test_two_steps_match_hand_worked_values():
    k = 2 * nn.N_IN + 3  # one trainable entry
    flat = np.zeros(NP)
    flat[k] = GOLD["w0"]
    m = np.zeros(NP)
    v = np.zeros(NP)
    for t, (g, ref) in enumerate(zip(GOLD["gradients"], (GOLD["step1"], GOLD["step2"])), start=1):
        grad = np.zeros(NP)
        grad[k] = g
        flat, m, v = nn.adam_update(flat, grad, m, v, t, GOLD["lr"], GOLD["b1"], GOLD["b2"],
                                    GOLD["eps"])
        assert m[k] == pytest.approx(ref["m"], rel=1e-14)
        assert v[k] == pytest.approx(ref["v"], rel=1e-14)
        assert flat[k] == pytest.approx(ref["w"], rel=1e-14, abs=0)
    others = np.ones(NP, bool)
    others[k] = False
    assert np.all(flat[others] == 0.0)


def test_constant_gradient_moves_each_step_by_lr_times_sign():
    rng = np.random.default_rng(1)
    g = rng.standard_normal(NP) * 10.0 ** rng.uniform(-4, 2, NP)
    flat0 = rng.standard_normal(NP)
    flat, m, v = flat0.copy(), np.zeros(NP), np.zeros(NP)
    lr, eps = 1e-3, 1e-8
    for t in range(1, 6):
        prev = flat.copy()
        flat, m, v = nn.adam_update(flat, g, m, v, t, lr, eps=eps)
        step = (prev - flat)[TRAINABLE]
        np.testing.assert_allclose(step, lr * g[TRAINABLE] / (np.abs(g[TRAINABLE]) + eps),
                                   rtol=1e-9, atol=0)
    np.testing.assert_array_equal(flat[:2 * nn.N_IN], flat0[:2 * nn.N_IN])
    np.testing.assert_array_equal(flat[-2:], flat0[-2:])


def test_first_step_is_scale_free():
    rng = np.random.default_rng(2)
    g = rng.standard_normal(NP)
    a = nn.adam_update(np.zeros(NP), g, np.zeros(NP), np.zeros(NP), 1, 0.01)[0]
    b = nn.adam_update(np.zeros(NP), 1e3 * g, np.zeros(NP), np.zeros(NP), 1, 0.01)[0]
    gt = g[TRAINABLE]
    np.testing.assert_allclose(-a[TRAINABLE], 0.01 * gt / (np.abs(gt) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(-b[TRAINABLE], 0.01 * gt / (np.abs(gt) + 1e-11), rtol=1e-12)
    np.testing.assert_allclose(np.abs(b[TRAINABLE]), 0.01, rtol=1e-7)
