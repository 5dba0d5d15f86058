"""Pins of the control-variate oracle (oracle/cv.py)."""
import numpy as np
import pytest

import oracle
from oracle import cv
from paper_2312_02990_gb300 import inputs


def rand_theta(seed, scale=0.2):
    return np.random.default_rng(seed).normal(0, scale, cv.N_PARAMS)


def test_parameter_count_is_32_128_128_1():
    assert cv.N_PARAMS == 20865


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    th = rand_theta(2)
    X = rng.normal(size=(7, cv.N_FEAT))
    y = rng.normal(size=7)
    loss, g = cv.backward(th, X, y)
    idx = rng.choice(cv.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [cv.N_PARAMS - 1, 0, cv.HIDDEN * cv.N_FEAT]])
    h = 1e-6
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h; tm[k] -= h
        fd = (cv.backward(tp, X, y)[0] - cv.backward(tm, X, y)[0]) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-6, abs=1e-10)


def test_forward_of_a_constant_network():
    W1 = np.zeros((128, 32)); b1 = np.full(128, np.arctanh(0.5))
    W2 = np.zeros((128, 128)); b2 = np.full(128, np.arctanh(0.25))
    W3 = np.ones(128); b3 = -3.0
    out, _ = cv.forward(cv.pack(W1, b1, W2, b2, W3, b3), np.random.default_rng(0).normal(size=(5, 32)))
    assert np.allclose(out, 128 * 0.25 - 3.0, rtol=1e-14)


def test_adam_first_step_moves_by_lr_times_sign():
    th = np.array([1.0, -2.0, 0.5]); g = np.array([3.0, -0.01, 1e-3])
    t1, m, v = cv.adam_step(th, g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    # |step| = lr |g| / (|g| + eps): lr up to a relative eps/|g|
    assert np.allclose(t1, th - 0.1 * np.sign(g), rtol=0, atol=0.1 * 1e-8 / 1e-3 * 1.01)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounds_to_nearest_even():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1.5, 3.0e-3, 65504.0], dtype=np.float32)
    r = cv.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2 ** -6 and r[3] == -1.5
    assert abs(r[4] - 3.0e-3) <= 2 ** -8 * 3.0e-3
    # values with 8 significant bits are exact
    e = np.array([1.0078125, 0.75, -96.0], dtype=np.float32)
    assert np.array_equal(cv.bf16(e), e.astype(np.float64))


def test_feature_sign_rules_match_explicitly_mapped_states():
    N = 256
    b = oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))
    st = inputs.jittered_states(N, 1, seed=31, amp=0.1)[0]
    raw = cv.raw_features(b, st)
    for m in range(4):
        ms, am = oracle.apply_mapping(b, m, st, 0.3)
        direct = cv.mapped_features(cv.raw_features(b, ms), am, 0, N, b.V)
        via_signs = cv.mapped_features(raw, 0.3, m, N, b.V)
        assert np.allclose(direct, via_signs, rtol=1e-10, atol=1e-13), m
    # stresses agree with the (independently pinned) pressure tensor
    P, U, K2 = oracle.pressure(b, st)
    f = cv.mapped_features(raw, 0.0, 0, N, b.V)
    assert np.allclose(f[0:6] + f[6:12], P, rtol=1e-12, atol=1e-14)
    assert f[12] == pytest.approx(U / N) and f[13] == pytest.approx(0.5 * K2 / N)
    assert f[15] == pytest.approx(P[3] ** 2)


def test_targets_of_linear_responses():
    t = np.arange(11) * 0.1
    B = np.stack([2 * t, -t])
    z = cv.targets(B, np.array([3.0, 4.0]), 0.5, 0.1)
    assert np.allclose(z, [3.0 * 1.0 / 0.5, 4.0 * (-0.5) / 0.5])


def test_cv_estimator_is_unbiased_and_reduces_variance_as_one_minus_rho2():
    rng = np.random.default_rng(7)
    mu, rho = 2.0, 0.9
    est, se_cv, se_pl = [], [], []
    for _ in range(400):
        xi_D = rng.normal(size=200)
        y = mu + rho * xi_D + np.sqrt(1 - rho ** 2) * rng.normal(size=200)
        h_M = rng.normal(size=20000)
        e, s, ep, sp = cv.cv_estimate(y, xi_D, h_M, rho)
        est.append(e); se_cv.append(s); se_pl.append(sp)
    est = np.array(est)
    assert abs(est.mean() - mu) < 3 * est.std(ddof=1) / np.sqrt(len(est))
    ratio = (np.mean(se_cv) / np.mean(se_pl)) ** 2
    assert ratio == pytest.approx(1 - rho ** 2 + rho ** 2 * 200 / 20000, rel=0.1)
    assert cv.fit_c(np.arange(10.0) * 3 + 1, np.arange(10.0)) == pytest.approx(3.0)
