"""mpdo_measure_1q_noalloc: the same observables as mpdo_measure_1q, computed
without any device allocation, on a state held in the caller's own device
memory.  It exists for callers that cannot call cudaMalloc (code running while
a stream is captured into a CUDA graph, frameworks that own all device memory
through their own pool); its scratch is a static device array shared by all
calls.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import build as B
    B.build()
    return torch


def _device_state(torch, s, batch, n, cap):
    """Copy the solver's state into caller-owned device tensors in libmpdo's layout."""
    sites = np.zeros((batch, n, cap, 4, cap))
    dims = np.zeros((batch, n + 1), np.int32)
    for b in range(batch):
        d, tens = s.get_state(b)
        dims[b] = d
        for p, t in enumerate(tens):
            sites[b, p, :t.shape[0], :, :t.shape[2]] = t
    return (torch.tensor(sites, device="cuda", dtype=torch.float64),
            torch.tensor(dims, device="cuda", dtype=torch.int32))


def test_noalloc_matches_measure_1q_twice(torch_cuda):
    torch = torch_cuda
    from paper_2203_05871_gb300 import Solver, load_library
    lib = load_library()
    n, batch, cap = 8, 2, 32
    wl = W.random_model(n, W.chain_bonds(n), 91, batch=batch, chi_max=cap, cutoff=1e-12)
    with Solver(n, batch=batch, chi_cap=cap) as s:
        s.build_gates(wl)
        s.step(3)
        ref = {c: s.measure_1q(range(n), c) for c in "ZX"}
        sites, dims = _device_state(torch, s, batch, n, cap)
    qubits = torch.arange(n, device="cuda", dtype=torch.int32)
    stream = torch.cuda.current_stream()
    for comp in "ZX":   # two calls in a row share the static scratch
        out = torch.full((batch, n), float("nan"), device="cuda", dtype=torch.float64)
        rc = lib.mpdo_measure_1q_noalloc(ctypes.c_void_p(sites.data_ptr()), ctypes.c_void_p(dims.data_ptr()), n,
                                         batch, cap, ctypes.c_void_p(qubits.data_ptr()), n, comp.encode(),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.mpdo_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref[comp]).max() <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_2203_05871_gb300 import load_library
    lib = load_library()
    buf = torch.zeros(16, device="cuda", dtype=torch.float64)
    ibuf = torch.zeros(16, device="cuda", dtype=torch.int32)
    p, ip = ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(ibuf.data_ptr())
    # 2 * 64 * 41 * 512 doubles > 2^18: rejected before any launch
    rc = lib.mpdo_measure_1q_noalloc(p, ip, 40, 64, 512, ip, 1, b"Z", p, None)
    assert rc == -7
    assert "static scratch" in lib.mpdo_last_error().decode()
