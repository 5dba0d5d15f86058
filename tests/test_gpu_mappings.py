"""GPU parity of the mappings beyond Eq. 3 (each position/momentum
component mirrored, x and z exchanged; mapping codes 0..31, codes 0..3 being
Eq. 3): the spawned B(0) = P_xy and Omega(0) of every mapped daughter, and
their first steps, against the oracle applying the same mapping explicitly.

Tolerances: B(0), Omega(0) relative 1e-11 (IEEE double on both sides, the
GPU forms them as sign flips of the mother's P_xy or P_zy, the oracle from
the mapped state); 30-step B(s) as in test_gpu_parity (FP64 1e-9, MIXED
1e-4 relative to the series' scale)."""
import numpy as np
import pytest

import oracle
from paper_2312_02990_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL = 0xFFFFFFFF


@pytest.fixture(scope="module")
def ttcf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_02990_gb300 import ttcf as T
    T.load(build_if_missing=True)
    return T


def ctx(T, **kw):
    c = T.config_default()
    for k, v in kw.items():
        setattr(c, k, v)
    return T.Context(c)


def test_spawn_of_every_mapping_matches_the_oracle(ttcf, eq_mothers_256):
    b, ms, al = eq_mothers_256
    G = 3
    gam = np.array([1e-2, 1e-4, 1e-6])
    with ctx(ttcf, precision=1, n_steps=2, mapping_mask=ALL) as c:
        bid = c.spawn_daughters(ms[:G], al[:G], gam, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 32 * G)
        om_mean, n_valid = c.omega_mean(bid)
    for g in range(G):
        for m in range(32):
            mo, _ = oracle.apply_mapping(b, m, ms[g], al[g])
            P = oracle.pressure(b, mo)[0][3]
            d = 32 * g + m
            assert B[d, 0] == pytest.approx(P, rel=1e-11, abs=1e-13), (g, m)
            assert Om[d] == pytest.approx(-gam[g] * b.V * P / b.T, rel=1e-11, abs=1e-13 * gam[g] * b.V), (g, m)
        # the set is closed under the x-reflection: exact cancellation
        assert Om[32 * g:32 * g + 32].sum() == 0.0
        assert B[32 * g:32 * g + 32, 0].sum() == 0.0
    assert om_mean == 0.0 and n_valid == G


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-4)])
def test_every_mapping_follows_the_oracle(ttcf, eq_mothers_256, precision, tol):
    b, ms, al = eq_mothers_256
    gamma, n = 0.02, 30
    with ctx(ttcf, precision=precision, n_steps=n, mapping_mask=ALL) as c:
        bid = c.spawn_daughters(ms[:1], al[:1], gamma, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 32)
    Bo, Omo = oracle.daughters(b, ms[:1], al[:1], gamma, n, mapping_mask=ALL)
    scale = np.abs(Bo).max()
    assert np.abs(B - Bo).max() < tol * scale
    assert np.allclose(Om, Omo, rtol=1e-11, atol=1e-13 * np.abs(Omo).max())


def test_a_subset_of_mappings_in_the_ensemble(ttcf, eq_mothers_256):
    """Eq. 3's four mappings with the z-mirror (8 codes) as one ensemble:
    responses equal the oracle's reduction of its own daughters (FP64, 60
    steps, where trajectories still agree closely)."""
    b, ms, al = eq_mothers_256
    mask, n, gamma = 0x0F0F, 60, 0.05
    with ctx(ttcf, precision=0, n_steps=n, mapping_mask=mask) as c:
        bid = c.spawn_daughters(ms[:6], al[:6], gamma, box=b.L)
        c.run()
        r = c.response(bid)
    Bo, Omo = oracle.daughters(b, ms[:6], al[:6], gamma, n, mapping_mask=mask)
    ro = oracle.responses(Bo, Omo, 8, b.dt)
    for k in ("corr", "dav", "ttcf"):
        assert np.allclose(r[k], ro[k], rtol=1e-6, atol=1e-9 * np.abs(ro[k]).max()), k


def test_exchange_needs_a_square_xz_box(ttcf):
    T = ttcf
    st = inputs.jittered_states(256, 1, seed=2)
    L = inputs.bulk_box(256)
    with ctx(T, precision=1, n_steps=2, mapping_mask=1 << 16) as c:
        with pytest.raises(T.TTCFError) as e:
            c.spawn_daughters(st, None, 0.1, box=(L[0], L[1], L[2] * 1.1))
        assert e.value.status == T.TTCF_E_INVALID
