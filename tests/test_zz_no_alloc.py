"""The allocation-free residual entry point, st_residual_noalloc, called through the C ABI.

Some callers cannot allocate device memory while they run: frameworks that own all device memory
through their own pool, and loops that cannot take cudaMalloc's implicit device synchronisation.
For them the library offers the FP64 residual with its scratch in a fixed device array.  These tests check it against st_residual on
the same inputs, twice in a row (the fixed array keeps the previous call's contents), within the
residual parity tolerance; that repeated calls change neither torch's allocator nor the device's
free memory; and that a size beyond the fixed array is refused.  The file is named to run after
every other test file.
"""
import ctypes
import gc

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,p,N,with_psi0", [(19, 2, 7, True), (33, 1, 17, False)])
def test_residual_noalloc_matches_residual(n, p, N, with_psi0):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07269_gb300 import _lib, build, stfdm

    build.build()
    L = _lib.lib()
    dev = torch.device("cuda:0")
    h = stfdm.setup_problem(n, p, synth.uniform_time_nodes(N, 1.2), device=0)
    x1, x2 = synth.interior_coords(n)
    psi0 = torch.from_numpy(synth.packet_values(synth.packet_params(3), x1, x2)).to(dev) if with_psi0 else None
    F = torch.from_numpy(synth.cn01((h.n_t, h.n_x), seed=n)).to(dev)
    for call in range(2):
        psi = torch.from_numpy(synth.cn01((h.n_t, h.n_x), seed=100 * n + call)).to(dev)
        R_ref = torch.empty_like(F)
        rel_ref, _ = stfdm.st_residual(h, F, psi0, psi, R_ref)
        R = torch.full_like(F, float("nan"))
        norms = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        st = L.st_residual_noalloc(h.ptr, ctypes.c_void_p(F.data_ptr()),
                                   ctypes.c_void_p(psi0.data_ptr()) if psi0 is not None else None,
                                   ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                   ctypes.c_void_p(norms.data_ptr()), stream)
        assert st == _lib.ST_OK
        torch.cuda.synchronize()
        Rn, Rr = R.cpu().numpy(), R_ref.cpu().numpy()
        scale = np.abs(F.cpu().numpy()).max()
        np.testing.assert_allclose(Rn, Rr, rtol=0, atol=1e-13 * scale)
        nr = norms.cpu().numpy()
        rel = float(np.sqrt(nr[0] / nr[1]))
        assert abs(rel - rel_ref) <= 1e-12 * rel_ref
        assert abs(nr[0] - float(np.sum(np.abs(Rr) ** 2))) <= 1e-12 * nr[0]


def test_residual_noalloc_allocates_nothing():
    """Through the Python wrapper: after one warm-up call (which looks up the fixed array's device
    address), two more calls leave torch's allocated bytes and the device's free bytes unchanged,
    and both agree with st_residual.  R aliasing psi is refused (other threads still read psi's
    stencil neighbours while R is written)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07269_gb300 import _lib, build, stfdm

    build.build()
    dev = torch.device("cuda:0")
    n, N = 41, 24
    h = stfdm.setup_problem(n, 1, synth.uniform_time_nodes(N, 1.0), device=0)
    x1, x2 = synth.interior_coords(n)
    psi0 = torch.from_numpy(synth.packet_values(synth.packet_params(5), x1, x2)).to(dev)
    F = torch.from_numpy(synth.cn01((h.n_t, h.n_x), seed=7)).to(dev)
    psis = [torch.from_numpy(synth.cn01((h.n_t, h.n_x), seed=8 + i)).to(dev) for i in range(2)]
    R = torch.empty_like(F)
    norms = torch.empty(2, dtype=torch.float64, device=dev)
    R_ref = torch.empty_like(F)
    got = [(torch.empty_like(F), torch.empty_like(norms)) for _ in psis]   # allocated before measuring
    stfdm.st_residual_noalloc(h, F, psi0, psis[0], R, norms)     # warm-up
    torch.cuda.synchronize()
    # tensors left for the garbage collector by earlier tests in this process would otherwise be
    # freed at a random point of the measured calls and change torch's count
    gc.collect()
    gc.disable()
    try:
        alloc0 = torch.cuda.memory_allocated(dev)
        free0, _ = torch.cuda.mem_get_info(dev)
        for psi, (Rg, ng) in zip(psis, got):
            stfdm.st_residual_noalloc(h, F, psi0, psi, R, norms)
            Rg.copy_(R)
            ng.copy_(norms)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(dev)
        alloc1 = torch.cuda.memory_allocated(dev)
    finally:
        gc.enable()
    assert alloc1 == alloc0
    assert free1 == free0
    for psi, (Rg, ng) in zip(psis, got):
        rel_ref, _ = stfdm.st_residual(h, F, psi0, psi, R_ref)
        scale = float(torch.abs(F).max())
        assert float(torch.abs(Rg - R_ref).max()) <= 1e-13 * scale
        nr = ng.cpu().numpy()
        assert abs(float(np.sqrt(nr[0] / nr[1])) - rel_ref) <= 1e-12 * rel_ref
    with pytest.raises(ValueError):
        stfdm.st_residual_noalloc(h, F, psi0, psis[0], psis[0], norms)
    L = _lib.lib()
    st = L.st_residual_noalloc(h.ptr, ctypes.c_void_p(F.data_ptr()), None, ctypes.c_void_p(R.data_ptr()),
                               ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(norms.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.ST_ERR_ARG


def test_residual_noalloc_rejects_too_large():
    """Above the fixed scratch (65,536 blocks of 256 nodes x 16 time rows) the call is refused
    with ST_ERR_ARG before any pointer is used.  4097 squares per direction give 4096^2 =
    16,777,216 interior nodes; with 17 time DOFs that is 65,536 x 2 blocks.  The size check comes
    first, so small placeholder buffers stand in for the space-time arrays."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07269_gb300 import _lib, build, stfdm

    build.build()
    L = _lib.lib()
    dev = torch.device("cuda:0")
    h = stfdm.setup_problem(4097, 1, synth.uniform_time_nodes(17, 1.0), device=0)
    assert h.n_x == 4096 * 4096
    assert ((h.n_x + 255) // 256) * ((h.n_t + 15) // 16) == 65536 * 2
    F = torch.zeros(16, dtype=torch.complex128, device=dev)
    psi = torch.zeros_like(F)
    norms = torch.zeros(2, dtype=torch.float64, device=dev)
    st = L.st_residual_noalloc(h.ptr, ctypes.c_void_p(F.data_ptr()), None, ctypes.c_void_p(psi.data_ptr()), None,
                               ctypes.c_void_p(norms.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.ST_ERR_ARG
    assert "fixed scratch" in L.st_last_error_message().decode()
