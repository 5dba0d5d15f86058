"""CPU checks of the C ABI: the library builds, loads and exports every
function declared in include/ttcf.h; without a GPU, creation fails cleanly."""
import ctypes as C
import os
import re

import pytest

from paper_2312_02990_gb300 import build as libbuild
from paper_2312_02990_gb300 import ttcf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ttcf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ttcf_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    path = libbuild.build()
    lib = C.CDLL(path)
    names = declared_functions()
    assert "ttcf_create" in names and "ttcf_run" in names and len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(ttcf.EXPORTS) == set(names)


def test_config_default_and_version():
    c = ttcf.config_default()
    assert (c.dt, c.T, c.tau_T, c.n_steps, c.sample_every, c.mapping_mask) == (0.0025, 0.722, 0.25, 1000, 1, 0xF)
    assert c.precision == ttcf.TTCF_MIXED
    assert "sm_103a" in ttcf.version()


def test_create_rejects_bad_configs_before_touching_the_gpu():
    L = ttcf.load()
    h = C.c_void_p()
    for field, val in (("dt", -1.0), ("n_steps", 0), ("sample_every", 3), ("mapping_mask", 0),
                       ("precision", 7), ("block_threads", 48), ("kernel_variant", 9)):
        c = ttcf.config_default()
        setattr(c, field, val)
        st = L.ttcf_create(C.byref(c), C.byref(h))
        assert st == ttcf.TTCF_E_INVALID, field
        assert L.ttcf_last_error(None)


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ttcf.TTCFError) as e:
        ttcf.Context(use_torch_allocator=False, torch_stream=False)
    assert e.value.status == ttcf.TTCF_E_CUDA


def test_null_handles_are_rejected():
    L = ttcf.load()
    assert L.ttcf_run(None, 10) == ttcf.TTCF_E_INVALID
    L.ttcf_destroy(None)
