"""The allocation-free V-cycle entry point (mg_op_vcycle_static) against the
allocating one (mg_op_vcycle), through the C ABI (GPU).

mg_op_vcycle_static exists for callers that cannot call cudaMalloc (a solver
stepped inside a fixed-rate loop that cannot take the device-wide
synchronisation of an allocation, or a process whose framework allocator has
reserved most of the device memory).  It keeps the coarsest-grid
pseudo-inverse in a static device array instead of allocating it.  This file
is collected last so that a run stopping at its first failure has already run
every other test; it passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg
    return mg.load()


def _case(n, dt, seed):
    rng = np.random.default_rng(seed)
    x0 = torch.tensor(rng.standard_normal((n, n)), dtype=dt, device=DEV)
    b = rng.standard_normal((n, n))
    b = torch.tensor(b - b.mean(), dtype=dt, device=DEV)
    return x0, b


def test_static_vcycle_matches_allocating_vcycle_on_two_calls(lib):
    stream = torch.cuda.current_stream().cuda_stream
    # (dtype code, torch dtype, n, coarsest, nu1, nu2, zero_init, tolerance)
    calls = [(0, torch.float64, 64, 8, 2, 2, 0, 1e-12),
             (1, torch.float32, 32, 16, 1, 2, 1, 2e-5)]
    outs = []
    for k, (code, dt, n, coarsest, nu1, nu2, zero, tol) in enumerate(calls):
        x0, b = _case(n, dt, 100 + k)
        x_static = x0.clone()
        st = lib.mg_op_vcycle_static(code, n, coarsest, C.c_void_p(x_static.data_ptr()),
                                     C.c_void_p(b.data_ptr()), nu1, nu2, zero, C.c_void_p(stream))
        assert st == 0, lib.mg_last_error()
        outs.append((x_static, x0, b, code, n, coarsest, nu1, nu2, zero, tol))
    torch.cuda.synchronize()  # both static calls queued back to back, then checked
    for x_static, x0, b, code, n, coarsest, nu1, nu2, zero, tol in outs:
        x_ref = x0.clone()
        st = lib.mg_op_vcycle(code, n, coarsest, C.c_void_p(x_ref.data_ptr()),
                              C.c_void_p(b.data_ptr()), nu1, nu2, zero, C.c_void_p(stream))
        assert st == 0, lib.mg_last_error()
        torch.cuda.synchronize()
        ref = x_ref.double().cpu().numpy()
        got = x_static.double().cpu().numpy()
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
        assert np.abs(got - x0.double().cpu().numpy()).max() > 0  # the cycle did run


def test_static_vcycle_rejects_sizes_beyond_its_scratch(lib):
    x = torch.zeros((128, 128), dtype=torch.float64, device=DEV)
    for n, coarsest in ((128, 8), (64, 32)):
        st = lib.mg_op_vcycle_static(0, n, coarsest, C.c_void_p(x.data_ptr()),
                                     C.c_void_p(x.data_ptr()), 2, 2, 1, None)
        assert st == 1  # MG_ERR_INVALID_ARG
        assert b"static scratch" in lib.mg_last_error()


def test_static_vcycle_neither_waits_nor_holds_memory(lib):
    """The call is asynchronous (it returns while earlier work on its stream
    is still running: no allocation or other device-wide synchronisation
    inside it) and leaves the device's free memory unchanged."""
    stream = torch.cuda.current_stream()
    x0, b = _case(64, torch.float64, 7)
    x = x0.clone()
    st = lib.mg_op_vcycle_static(0, 64, 8, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()), 2, 2, 0,
                                 C.c_void_p(stream.cuda_stream))
    assert st == 0, lib.mg_last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    torch.cuda._sleep(200_000_000)  # ~0.1 s of spinning on the stream
    st = lib.mg_op_vcycle_static(0, 64, 8, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()), 2, 2, 0,
                                 C.c_void_p(stream.cuda_stream))
    busy = not stream.query()
    assert st == 0, lib.mg_last_error()
    assert busy  # returned before the sleep ahead of it finished
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0



def test_static_vcycle_records_into_a_cuda_graph(lib):
    """The call can be captured into a CUDA graph (global capture mode, in
    which an allocation or a device-wide synchronisation inside the call would
    make the capture fail); each replay gives the bits of an uncaptured call."""
    x0, b = _case(64, torch.float64, 11)
    side = torch.cuda.Stream()
    x_ref = x0.clone()
    st = lib.mg_op_vcycle_static(0, 64, 8, C.c_void_p(x_ref.data_ptr()), C.c_void_p(b.data_ptr()), 2, 2, 0,
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.mg_last_error()
    torch.cuda.synchronize()
    x = x0.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        st = lib.mg_op_vcycle_static(0, 64, 8, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()), 2, 2, 0,
                                     C.c_void_p(side.cuda_stream))
    assert st == 0, lib.mg_last_error()
    for _ in range(2):
        x.copy_(x0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(x, x_ref)
