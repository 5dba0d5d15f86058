"""GPU control variate (not in the paper; the estimator it improves is
Eq. 1) against the FP64 oracle of oracle/cv.py.

Tolerances: features 1e-5 relative (FP32 features kernel against FP64
sums); targets 1e-12 relative (FP64 on both sides); network outputs and
gradients with the BF16-rounded weights on both sides, FP32 accumulation on
the GPU (the forward pass on the tensor cores with the activations as two
BF16 terms, about 2^-17 relative per product): 1e-4 relative to the
largest entry."""
import numpy as np
import pytest

import oracle
from oracle import cv as ocv
from paper_2312_02990_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_02990_gb300 import ttcf
    ttcf.load(build_if_missing=True)
    return ttcf


def ctx(T, **kw):
    c = T.config_default()
    for k, v in kw.items():
        setattr(c, k, v)
    return T.Context(c)


def test_features_and_targets_match_the_oracle(T, eq_mothers_256):
    b, ms, al = eq_mothers_256
    G, n, gamma = 6, 60, 1e-3
    with ctx(T, precision=0, n_steps=n) as c:
        bid = c.spawn_daughters(ms[:G], al[:G], gamma, box=b.L)
        c.run()
        X, z = c.cv_data(bid, 4 * G)
        B, Om = c.daughter_series(bid, 4 * G)
    zo = ocv.targets(B, Om, gamma, b.dt)
    assert np.allclose(z, zo, rtol=1e-12, atol=0)
    for g in range(G):
        raw = ocv.raw_features(b, ms[g])
        for m in range(4):
            xo = ocv.mapped_features(raw, al[g], m, b.n, b.V)
            assert np.allclose(X[4 * g + m], xo, rtol=1e-5, atol=1e-6 * np.abs(xo).max()), (g, m)


def test_forward_and_gradient_match_the_oracle(T):
    rng = np.random.default_rng(3)
    th = rng.normal(0, 0.15, ocv.N_PARAMS).astype(np.float32)
    X = rng.normal(size=(77, 32)).astype(np.float32)
    y = rng.normal(size=77).astype(np.float32)
    thb = ocv.bf16(th)   # the GPU computes with the BF16 rounding of the weights
    with ctx(T) as c:
        f = c.cv_forward(th, X)
        g, loss = c.cv_gradient(th, X, y)
    fo, _ = ocv.forward(thb, X.astype(np.float64))
    lo, go = ocv.backward(thb, X.astype(np.float64), y.astype(np.float64))
    assert np.abs(f - fo).max() < 1e-4 * np.abs(fo).max()
    assert loss == pytest.approx(lo, rel=1e-4)
    assert np.abs(g - go).max() < 1e-4 * np.abs(go).max()


def test_tensor_core_forward_over_many_tiles(T):
    """The forward pass runs on the tensor cores (tcgen05, 128 samples per
    tile, activations as two BF16 terms, FP32 accumulation in tensor memory):
    40001 samples (many tiles per CTA and a ragged last tile) against the
    FP64 oracle with the same BF16 weights, 1e-4 of the largest output."""
    rng = np.random.default_rng(17)
    th = rng.normal(0, 0.12, ocv.N_PARAMS).astype(np.float32)
    X = rng.normal(size=(40001, 32)).astype(np.float32)
    with ctx(T) as c:
        f = c.cv_forward(th, X)
    fo, _ = ocv.forward(ocv.bf16(th), X.astype(np.float64))
    assert np.all(np.isfinite(f))
    assert np.abs(f - fo).max() < 1e-4 * np.abs(fo).max()
    # the outputs also follow the inputs row by row (no tile or row mix-up)
    assert np.corrcoef(f, fo)[0, 1] > 0.999999


def test_control_variate_is_unbiased_and_reduces_variance(T):
    """Config-1 system: train on daughters at gamma = 1e-3, evaluate at
    gamma = 1e-6 on disjoint mothers, with an independent auxiliary set of
    16x as many mother states (features only).  The variance factor of the
    estimator is 1 - rho^2 + rho^2 |D|/|M| (oracle pin), so the auxiliary
    set must be much larger than D for any gain."""
    N = 256
    L = inputs.bulk_box(N)
    nD = 512
    with ctx(T, precision=1, n_steps=400) as c:
        init = np.stack([inputs.initial_state(N, 500 + k) for k in range(64)])
        ms, al = c.sample_mothers(init, L, n_eq=4000, n_states=160, spacing=150)
        ms, al = ms.reshape(-1, 6, N), al.reshape(-1)
        # interleave the independent mothers so each set spans all of them
        order = np.arange(ms.shape[0]).reshape(64, 160).T.ravel()
        ms, al = ms[order], al[order]
        tr, ev, aux = slice(0, 1536), slice(1536, 1536 + nD), slice(1536 + nD, 1536 + 17 * nD)
        bt = c.spawn_daughters(ms[tr], al[tr], 1e-3, box=L)
        be = c.spawn_daughters(ms[ev], al[ev], 1e-6, box=L)
        c.run()
        cfg = T.cv_config_default()
        cfg.epochs = 25
        loss = c.cv_train(bt, cfg)
        r = c.cv_apply(be, ms[aux], al[aux])
        # the same auxiliary states from device memory give the same numbers
        import torch
        rd = c.cv_apply(be, torch.from_numpy(np.ascontiguousarray(ms[aux])).cuda(),
                        torch.from_numpy(np.ascontiguousarray(al[aux])).cuda())
        v = c.viscosity(be)
    assert rd == r
    assert loss[-1] < 0.9 * loss[0]
    assert r["n_groups"] == nD and r["n_aux"] == 16 * nD
    assert r["eta_plain"] == pytest.approx(v["eta_ttcf"][-1], rel=1e-9)
    assert r["se_plain"] == pytest.approx(v["eta_ttcf_se"][-1], rel=1e-9)
    assert abs(r["eta_cv"] - r["eta_plain"]) < 2.0 * np.hypot(r["se_cv"], r["se_plain"])
    assert r["gain"] > 1.0, r
    print("control variate:", r)
