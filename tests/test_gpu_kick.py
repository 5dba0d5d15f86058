"""GPU parity of the momentum kicks (ttcf_kick_states) through the C ABI
against the oracle (oracle/kick.py) on the same inputs and seeds.

Tolerances: positions bit for bit (copied); momenta within 1e-12 of the
largest momentum (both sides IEEE double: the kicks differ by the last
bits of log, cos and sin and the group sums by their summation order).
"""
import numpy as np
import pytest

from oracle import kick as ok
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


def ctx(mod, **kw):
    c = mod.config_default()
    for k, v in kw.items():
        setattr(c, k, v)
    return mod.Context(c)


def close(a, b):
    scale = np.abs(b[:, 3:]).max()
    assert np.array_equal(a[:, :3], b[:, :3])
    assert np.abs(a[:, 3:] - b[:, 3:]).max() <= 1e-12 * scale


@pytest.mark.parametrize("keep_energy", [True, False])
def test_bulk_kicks_match_oracle(T, eq_mothers_256, keep_energy):
    b, ms, al = eq_mothers_256
    seed = 0xFEDCBA9876543210
    with ctx(T, T=0.722) as c:
        got = c.kick_states(ms[0], 5, 1e-2, seed, keep_energy=keep_energy)
    ref = ok.kick_states(ms[0], 5, 1e-2, 0.722, seed, keep_energy=keep_energy)
    close(got, ref)


def test_confined_groups_on_device(T):
    torch = pytest.importorskip("torch")
    s = inputs.confined_system(nx=10, nz=10, layers=2, seed=3)
    st, types = s["state"], s["types"]
    with ctx(T, system=T.TTCF_CONFINED_LJ, T=1.0) as c:
        got = c.kick_states(torch.from_numpy(st).cuda(), 3, 3e-2, 12345, types=types).cpu().numpy()
    ref = ok.kick_states(st, 3, 3e-2, 1.0, 12345, types=types, keep_energy=True)
    close(got, ref)
    for t in (0, 1, 2):   # each group keeps its net momentum and kinetic energy
        sel = types == t
        p0 = st[3:][:, sel]
        for k in range(3):
            p1 = got[k, 3:][:, sel]
            assert np.allclose(p1.sum(axis=1), p0.sum(axis=1), rtol=0, atol=1e-11)
            q0 = p0 - p0.mean(axis=1, keepdims=True)
            q1 = p1 - p1.mean(axis=1, keepdims=True)
            assert np.sum(q1 * q1) == pytest.approx(np.sum(q0 * q0), rel=1e-12)


def test_seeds_and_determinism(T, eq_mothers_256):
    b, ms, al = eq_mothers_256
    with ctx(T) as c:
        a1 = c.kick_states(ms[1], 2, 1e-3, 7)
        a2 = c.kick_states(ms[1], 2, 1e-3, 7)
        a3 = c.kick_states(ms[1], 2, 1e-3, 8)
    assert np.array_equal(a1, a2)
    assert not np.array_equal(a1[:, 3:], a3[:, 3:])
    assert not np.array_equal(a1[0, 3:], a1[1, 3:])


def test_invalid_kicks_are_rejected(T, eq_mothers_256):
    b, ms, al = eq_mothers_256
    bad_types = np.zeros(ms.shape[2], dtype=np.int32)
    bad_types[5] = 3
    with ctx(T) as c:
        for kw in (dict(kick=-1.0), dict(kick=float("nan")), dict(types=bad_types)):
            args = dict(n_copies=2, kick=1e-3, seed=1, types=None)
            args.update(kw)
            with pytest.raises(T.TTCFError) as e:
                c.kick_states(ms[0], **args)
            assert e.value.status == T.TTCF_E_INVALID
        with pytest.raises(T.TTCFError):
            c.kick_states(ms[0], 0, 1e-3, 1)


def test_kicked_copies_decorrelate(T, eq_mothers_256):
    """Copies kicked by 1e-6 sqrt(T) start with the same P_xy to ~1e-5 and,
    the dynamics being chaotic, end as independent samples: their spread
    reaches the equilibrium spread of P_xy."""
    b, ms, al = eq_mothers_256
    n, steps = 32, 5000
    with ctx(T, precision=T.TTCF_MIXED) as c:
        cp = c.kick_states(ms[0], n, 1e-6, 99)
        r = c.mother_acf(cp, b.L, n_eq=0, n_steps=steps, max_lag=10, want_series=True)
    ser = r["series"]                       # [n, steps]
    eq_sd = ser[:, -1000:].std()
    first = ser[:, :10].std(axis=0).max()
    last = ser[:, -200:].std(axis=0).mean()
    assert first < 1e-3 * eq_sd
    assert last > 0.6 * eq_sd
