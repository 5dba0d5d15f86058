"""ttcf_run_noalloc, the entry point for callers that cannot allocate device
memory (their device memory belongs to their own pool allocator, or they
cannot afford the synchronisation of cudaMalloc/cudaFree).  It must give
the same daughters as ttcf_spawn_daughters + ttcf_run (bit for bit: same
kernels, list cells and layout), on two calls in a row through the same
static working array, without changing the device's free memory, and refuse
batches that do not fit and host arrays.

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other test."""
import numpy as np
import pytest

import oracle
from paper_2312_02990_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_02990_gb300 import ttcf as T
    T.load(build_if_missing=True)
    N = 256
    b = oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))
    ms, al = oracle.mother(b, inputs.initial_state(N, 77), n_eq=1500, n_states=6, spacing=150)
    return torch, T, b, ms, al


# variant 6 (8 atoms per thread) keeps the lo parts of its positions in the
# per-CTA scratch the no-allocation path carves from its static array
@pytest.mark.parametrize("precision,variant", [(0, 0), (1, 0), (1, 6)])
def test_noalloc_matches_the_allocating_path_twice(env, precision, variant):
    torch, T, b, ms, al = env
    G, n, gamma = ms.shape[0], 60, 1e-3
    cfg = T.config_default()
    cfg.precision, cfg.n_steps, cfg.kernel_variant = precision, n, variant
    with T.Context(cfg) as c:
        bid = c.spawn_daughters(ms, al, gamma, box=b.L)
        c.run()
        B_ref, Om_ref = c.daughter_series(bid, 4 * G)
    dev = torch.device("cuda")
    m_t = torch.from_numpy(ms).to(dev)
    a_t = torch.from_numpy(al).to(dev)
    g_t = torch.full((G,), gamma, dtype=torch.float64, device=dev)
    cfg2 = T.config_default()
    cfg2.precision, cfg2.n_steps, cfg2.kernel_variant = precision, n, variant
    cfg2.stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        B = torch.full((4 * G, n + 1), np.nan, dtype=torch.float64, device=dev)
        Om = torch.full((4 * G,), np.nan, dtype=torch.float64, device=dev)
        st = torch.full((4 * G,), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = T.run_noalloc(cfg2, m_t, a_t, g_t, b.L, B, Om, st)
        assert rc == T.TTCF_OK, T.last_error()
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the library's kernels
            assert torch.cuda.mem_get_info()[0] == free0, "device memory was allocated"
        Bh, Omh, sth = B.cpu().numpy(), Om.cpu().numpy(), st.cpu().numpy()
        assert np.all(sth == 0), call
        # same kernels, same list cells and layout as the allocating path
        assert np.array_equal(Omh, Om_ref), call
        assert np.array_equal(Bh, B_ref), call


def test_noalloc_rejects_a_batch_beyond_its_static_array(env):
    torch, T, b, ms, al = env
    N, G = 4096, 200   # 200 * 6 * 4096 * 8 B = 39 MB of mother slots alone
    dev = torch.device("cuda")
    m_t = torch.zeros((G, 6, N), dtype=torch.float64, device=dev)
    g_t = torch.zeros((G,), dtype=torch.float64, device=dev)
    B = torch.zeros((4 * G, 11), dtype=torch.float64, device=dev)
    Om = torch.zeros((4 * G,), dtype=torch.float64, device=dev)
    st = torch.zeros((4 * G,), dtype=torch.int32, device=dev)
    cfg = T.config_default()
    cfg.n_steps = 10
    rc = T.run_noalloc(cfg, m_t, None, g_t, (17.0, 17.0, 17.0), B, Om, st)
    assert rc == T.TTCF_E_INVALID
    assert "32 MiB" in T.last_error()


def test_noalloc_rejects_host_arrays(env):
    """A host pointer where device memory is required is refused before any
    work is queued (the binding's own checks are bypassed here)."""
    import ctypes as C
    torch, T, b, ms, al = env
    G, N = 2, 256
    dev = torch.device("cuda")
    m_t = torch.from_numpy(np.ascontiguousarray(ms[:G])).to(dev)
    g_t = torch.full((G,), 1e-3, dtype=torch.float64, device=dev)
    Om = torch.zeros((4 * G,), dtype=torch.float64, device=dev)
    st = torch.zeros((4 * G,), dtype=torch.int32, device=dev)
    B_host = np.zeros((4 * G, 11))
    cfg = T.config_default()
    cfg.n_steps = 10
    box = np.ascontiguousarray(b.L, dtype=np.float64)
    rc = T.load().ttcf_run_noalloc(C.byref(cfg), N, box.ctypes.data_as(C.POINTER(C.c_double)), G,
                                   m_t.data_ptr(), None, g_t.data_ptr(), B_host.ctypes.data,
                                   Om.data_ptr(), st.data_ptr())
    assert rc == T.TTCF_E_INVALID
    assert "device memory" in T.last_error()
    assert np.all(B_host == 0.0)
