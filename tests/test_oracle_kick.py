"""Pins of the momentum-kick oracle (oracle/kick.py): the Philox-4x32-10
generator against its published known-answer vectors, the uniform and
Box-Muller transforms against their closed forms and the normal law, and
the conservation laws the kicked copies are defined to keep."""
import json
import os

import numpy as np
import pytest

from oracle import kick
from paper_2312_02990_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.json")


def test_philox_known_answers():
    kat = json.load(open(GOLDEN))
    for v in kat["vectors"]:
        ctr = np.array([[int(x, 16) for x in v["counter"]]], dtype=np.uint32)
        key = tuple(int(x, 16) for x in v["key"])
        out = kick.philox4x32_10(ctr, key)[0]
        assert [int(x) for x in out] == [int(x, 16) for x in v["out"]]


def test_uniform_ends_and_midpoint():
    z = np.array([0], dtype=np.uint32)
    f = np.array([0xFFFFFFFF], dtype=np.uint32)
    h = np.array([0x80000000], dtype=np.uint32)
    assert kick.uniform53(z, z)[0] == 2.0 ** -54
    assert kick.uniform53(f, f)[0] == 1.0 - 2.0 ** -54
    assert kick.uniform53(h, z)[0] == 0.5 + 2.0 ** -54


def test_gaussians_are_standard_normal():
    n = 200_000
    g = kick.gaussians(n, 3, 20231205)
    for k in range(3):
        x = g[k]
        assert abs(x.mean()) < 5 / np.sqrt(n)
        assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n)
        assert abs(np.mean(x ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)
        assert abs(np.mean(np.abs(x) < 1.0) - 0.682689492137) < 5 * np.sqrt(0.22 / n)
    # the components are uncorrelated, and copies differ
    assert abs(np.mean(g[0] * g[1])) < 5 / np.sqrt(n)
    assert abs(np.mean(g[0] * g[2])) < 5 / np.sqrt(n)
    h = kick.gaussians(n, 4, 20231205)
    assert abs(np.mean(g[0] * h[0])) < 5 / np.sqrt(n)


def test_box_muller_closed_form():
    """One counter by hand: the two words of each pair give u, and the pair
    of normals is sqrt(-2 ln u_a) (cos, sin)(2 pi u_b)."""
    seed, i, c = 0x0123456789ABCDEF, 7, 2
    w = kick.philox4x32_10(np.array([[i, c, 0, 0]], dtype=np.uint32),
                           (seed & 0xFFFFFFFF, seed >> 32))[0]
    ua = (((int(w[0]) << 32) | int(w[1])) >> 11) / 2.0 ** 53 + 2.0 ** -54
    ub = (((int(w[2]) << 32) | int(w[3])) >> 11) / 2.0 ** 53 + 2.0 ** -54
    g = kick.gaussians(8, c, seed)[:, i]
    r = np.sqrt(-2.0 * np.log(ua))
    assert g[0] == r * np.cos(2.0 * np.pi * ub)
    assert g[1] == r * np.sin(2.0 * np.pi * ub)


@pytest.mark.parametrize("keep_energy", [True, False])
def test_groups_keep_momentum_and_energy(keep_energy):
    s = inputs.confined_system(nx=10, nz=10, layers=2, seed=3)
    st, types = s["state"], s["types"]
    out = kick.kick_states(st, 3, 1e-2, 1.0, 99, types=types, keep_energy=keep_energy)
    assert out.shape == (3,) + st.shape
    assert np.array_equal(out[:, :3], np.repeat(st[None, :3], 3, axis=0))
    for c in range(3):
        assert not np.array_equal(out[c, 3:], st[3:])
        for t in (0, 1, 2):
            sel = types == t
            p0, p1 = st[3:][:, sel], out[c, 3:][:, sel]
            assert np.allclose(p1.sum(axis=1), p0.sum(axis=1), rtol=0, atol=1e-11)
            k0 = np.sum((p0 - p0.mean(axis=1, keepdims=True)) ** 2)
            k1 = np.sum((p1 - p1.mean(axis=1, keepdims=True)) ** 2)
            if keep_energy:
                assert k1 == pytest.approx(k0, rel=1e-12)
            else:
                assert k1 != pytest.approx(k0, rel=1e-6)


def test_kick_size_and_zero_kick():
    N = 2048
    st = inputs.initial_state(N, 5)
    T = 0.722
    # without the energy rescaling the change is the kick minus its mean
    out = kick.kick_states(st, 2, 1e-3, T, 7, keep_energy=False)
    d = out[0, 3:] - st[3:]
    assert abs(d.std() / (1e-3 * np.sqrt(T)) - 1.0) < 5 * np.sqrt(1.0 / (2 * 3 * N))
    assert np.allclose(d.sum(axis=1), 0.0, atol=1e-12)
    # a zero kick returns the state (up to the rounding of pbar + (p - pbar))
    z = kick.kick_states(st, 2, 0.0, T, 7, keep_energy=True)
    assert np.array_equal(z[1, :3], st[:3])
    assert np.abs(z[1, 3:] - st[3:]).max() < 1e-13 * np.abs(st[3:]).max()
