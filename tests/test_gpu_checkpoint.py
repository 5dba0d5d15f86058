"""Checkpoints (ttcf_save / ttcf_load) through the C ABI: a run interrupted,
written to disk and continued in a new context gives bitwise the series of
an uninterrupted run; a finished run reloads with identical responses."""
import ctypes
import struct

import numpy as np
import pytest

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


@pytest.mark.parametrize("precision", [0, 1])
def test_interrupted_run_continues_bitwise(T, eq_mothers_256, tmp_path, precision):
    b, ms, al = eq_mothers_256
    G, n = 8, 300
    gam = np.geomspace(1e-2, 1e-6, G)
    kw = dict(precision=precision, n_steps=n)
    with ctx(T, **kw) as c:
        bid = c.spawn_daughters(ms[:G], al[:G], gam, box=b.L)
        c.run()
        B_ref, Om_ref = c.daughter_series(bid, 4 * G)
        r_ref = c.response(bid)
    path = str(tmp_path / "run.ckpt")
    with ctx(T, **kw) as c:
        c.spawn_daughters(ms[:G], al[:G], gam, box=b.L)
        c.run(120)
        c.save(path)
    with ctx(T, **kw) as c:
        c.load(path)
        c.run()
        B, Om = c.daughter_series(0, 4 * G)
        r = c.response(0)
    assert np.array_equal(B, B_ref) and np.array_equal(Om, Om_ref)
    for k in ("corr", "dav", "ttcf", "ttcf_se"):
        assert np.array_equal(r[k], r_ref[k])


def test_finished_runs_reload_with_their_responses(T, eq_mothers_256, tmp_path):
    b, ms, al = eq_mothers_256
    path = str(tmp_path / "done.ckpt")
    with ctx(T, n_steps=100) as c:
        b1 = c.spawn_daughters(ms[:4], al[:4], 1e-3, box=b.L)
        b2 = c.spawn_daughters(ms[4:10], al[4:10], 1e-1, box=b.L)
        c.run()
        ref = [c.response(b1), c.viscosity(b2)]
        c.save(path)
    with ctx(T, n_steps=100) as c:
        c.load(path)
        got = [c.response(0), c.viscosity(1)]
        c.run()   # nothing left to run
    for k in ref[0]:
        assert np.array_equal(got[0][k], ref[0][k])
    for k in ref[1]:
        assert np.array_equal(got[1][k], ref[1][k])


def test_confined_run_reloads(T, tmp_path):
    s = inputs.confined_system(nx=10, nz=10, layers=2, seed=3)
    cfg = dict(system=T.TTCF_CONFINED_LJ, precision=T.TTCF_MIXED, dt=0.005, T=1.0, n_steps=20)
    path = str(tmp_path / "conf.ckpt")
    with ctx(T, **cfg) as c:
        bid = c.spawn_confined(s["state"][None], s["types"], s["lattice"], s["box"], None, 0.05)
        c.run()
        ref = c.response_obs(bid, 1)
        c.save(path)
    with ctx(T, **cfg) as c:
        c.load(path)
        got = c.response_obs(0, 1)
    for k in ref:
        assert np.array_equal(got[k], ref[k], equal_nan=True)


def test_checkpoint_errors(T, eq_mothers_256, tmp_path):
    b, ms, al = eq_mothers_256
    path = str(tmp_path / "a.ckpt")
    with ctx(T, n_steps=40) as c:
        c.spawn_daughters(ms[:2], al[:2], 1e-3, box=b.L)
        c.run(10)
        c.save(path)
    with ctx(T, n_steps=41) as c:          # another configuration
        with pytest.raises(T.TTCFError) as e:
            c.load(path)
        assert e.value.status == T.TTCF_E_INVALID
    with ctx(T, n_steps=40) as c:          # a used context
        c.spawn_daughters(ms[:2], al[:2], 1e-3, box=b.L)
        with pytest.raises(T.TTCFError) as e:
            c.load(path)
        assert e.value.status == T.TTCF_E_STATE
    junk = tmp_path / "junk.ckpt"
    junk.write_bytes(b"not a checkpoint at all")
    with ctx(T, n_steps=40) as c:
        with pytest.raises(T.TTCFError) as e:
            c.load(str(junk))
        assert e.value.status == T.TTCF_E_INVALID
    trunc = tmp_path / "trunc.ckpt"
    trunc.write_bytes(open(path, "rb").read()[:300])
    with ctx(T, n_steps=40) as c:
        with pytest.raises(T.TTCFError) as e:
            c.load(str(trunc))
        assert e.value.status == T.TTCF_E_INVALID


def test_tampered_header_is_rejected(T, eq_mothers_256, tmp_path):
    """A checkpoint whose cell count disagrees with its cell grid (the
    kernels index shared memory with it) is refused, not run."""
    b, ms, al = eq_mothers_256
    path = tmp_path / "t.ckpt"
    with ctx(T, n_steps=40) as c:
        c.spawn_daughters(ms[:2], al[:2], 1e-3, box=b.L)
        c.run(10)
        c.save(str(path))
    raw = bytearray(path.read_bytes())
    maps_bytes = 4 * 32   # the batch's table of mapping codes (32 int slots)
    off = 8 + 4 + ctypes.sizeof(T.Config) + 4 + 8 + 4 + 6 * 4 + maps_bytes + 24 + 24 + 12   # ncell
    ncell = struct.unpack_from("<i", raw, off)[0]
    nc = struct.unpack_from("<3i", raw, off - 12)
    assert ncell == nc[0] * nc[1] * nc[2]
    struct.pack_into("<i", raw, off, ncell + 7)
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    with ctx(T, n_steps=40) as c:
        with pytest.raises(T.TTCFError) as e:
            c.load(str(bad))
        assert e.value.status == T.TTCF_E_INVALID
