"""Equilibrium correlations along GPU mother trajectories (ttcf_mother_acf)
through the C ABI: the recorded P_xy follows the oracle's zero-field
trajectory for its first steps (MIXED tolerance as in test_gpu_parity), the
device autocorrelations equal the oracle's on the device series, and the
Green-Kubo integral equals the oracle's trapezoid integral times V/T."""
import numpy as np
import pytest

import oracle
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


def test_series_follows_the_oracle(T, eq_mothers_256):
    b, ms, al = eq_mothers_256
    n = 40
    with T.Context(T.config_default()) as c:
        r = c.mother_acf(ms[:1], b.L, n_eq=0, n_steps=n, max_lag=5, want_series=True)
    _, _, _, obs = oracle.trajectory(b, ms[0], n, gamma=0.0, alpha=0.0)
    pxy = obs[1:, 4]
    assert np.abs(r["series"][0] - pxy).max() < 1e-4 * np.sqrt(np.mean(pxy ** 2))


def test_correlations_match_their_definition(T):
    N = 256
    L = inputs.bulk_box(N)
    init = np.stack([inputs.initial_state(N, inputs.BASE_SEED + 300 + k) for k in range(4)])
    n, lag = 3000, 200
    with T.Context(T.config_default()) as c:
        r = c.mother_acf(init, L, n_eq=2000, n_steps=n, max_lag=lag, want_series=True)
    B = r["series"]
    acf, acf2 = oracle.autocorrelation(B, lag)
    assert np.allclose(r["acf_pxy"], acf, rtol=1e-10, atol=1e-14 * acf[0])
    assert np.allclose(r["acf_pxy2"], acf2, rtol=1e-9, atol=1e-12 * acf2[0])
    gk = oracle.green_kubo(acf, float(np.prod(L)), 0.722, 0.0025)
    assert np.allclose(r["eta_gk"], gk, rtol=1e-10, atol=1e-14)
    # an equilibrium stress correlation: largest at lag 0, decays within a
    # fraction of a time unit
    assert r["acf_pxy"][0] > 0 and np.abs(r["acf_pxy"][100:]).max() < 0.3 * r["acf_pxy"][0]
