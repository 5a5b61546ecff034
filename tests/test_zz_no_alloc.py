"""mpdo_measure_1q_noalloc: the same observables as mpdo_measure_1q, computed
without any device allocation, on a state held in the caller's own device
memory.  It serves callers that cannot call cudaMalloc, such as frameworks
that hand all device memory to their own pool up front; its scratch is a
static device array shared by all calls.  This file is collected last on
purpose."""
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
    """Copy the solver's state into caller-owned device tensors in the
    [batch][n][chi_cap][4][chi_cap] f64 layout the entry point reads."""
    sites = np.zeros((batch, n, cap, 4, cap))
    dims = np.zeros((batch, n + 1), np.int32)
    for b in range(batch):
        d, tens = s.get_state(b)
        dims[b] = d
        for p, t in enumerate(tens):
            sites[b, p, :t.shape[0], :, :t.shape[2]] = t
    return (torch.tensor(sites, device="cuda", dtype=torch.float64),
            torch.tensor(dims, device="cuda", dtype=torch.int32))


def _call(lib, torch, sites, dims, n, batch, cap, qubits, comp):
    out = torch.full((batch, qubits.numel()), 7.0, device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream()
    rc = lib.mpdo_measure_1q_noalloc(ctypes.c_void_p(sites.data_ptr()), ctypes.c_void_p(dims.data_ptr()), n,
                                     batch, cap, ctypes.c_void_p(qubits.data_ptr()), qubits.numel(), comp.encode(),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.mpdo_last_error().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _evolved(n, batch, cap, steps=3):
    from paper_2203_05871_gb300 import Solver
    wl = W.random_model(n, W.chain_bonds(n), 91, batch=batch, chi_max=cap, cutoff=1e-12)
    s = Solver(n, batch=batch, chi_cap=cap)
    s.build_gates(wl)
    s.step(steps)
    return wl, s


def test_noalloc_matches_measure_1q_twice(torch_cuda):
    torch = torch_cuda
    from paper_2203_05871_gb300 import load_library
    lib = load_library()
    n, batch, cap = 8, 2, 32
    _, s = _evolved(n, batch, cap)
    with s:
        ref = {c: s.measure_1q(range(n), c) for c in "ZX"}
        sites, dims = _device_state(torch, s, batch, n, cap)
    qubits = torch.arange(n, device="cuda", dtype=torch.int32)
    for comp in "ZX":   # two calls in a row share the static scratch
        got = _call(lib, torch, sites, dims, n, batch, cap, qubits, comp)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref[comp]).max() <= TOL


def test_noalloc_matches_the_oracle(torch_cuda):
    """The same state evolved by the CPU oracle (with the GPU's ranks): the
    allocation-free call reproduces its <sigma^z> and <sigma^y> directly."""
    torch = torch_cuda
    from oracle import tebd
    from paper_2203_05871_gb300 import load_library
    lib = load_library()
    n, batch, cap, steps = 7, 1, 16, 4
    wl, s = _evolved(n, batch, cap, steps)
    with s:
        ks = [int(k) for k in s.rank_log(steps)[0]]
        sites, dims = _device_state(torch, s, batch, n, cap)
    o = tebd.TEBD(wl).run(steps, forced_k=ks)
    qubits = torch.arange(n, device="cuda", dtype=torch.int32)
    for comp in "ZY":
        got = _call(lib, torch, sites, dims, n, batch, cap, qubits, comp)[0]
        want = np.array([o.state.expect_1q(i, comp) for i in range(n)])
        assert np.abs(got - want).max() <= TOL


def test_noalloc_out_of_range_dims_and_qubits_give_nan(torch_cuda):
    """Bond dimensions and qubits live in device memory, so the entry point
    clamps them on the device: an instance with a bond dimension above chi_cap
    and a qubit index >= n get NaN, everything else is still exact, and the
    next valid call is unaffected."""
    torch = torch_cuda
    from paper_2203_05871_gb300 import load_library
    lib = load_library()
    n, batch, cap = 8, 3, 32
    _, s = _evolved(n, batch, cap)
    with s:
        ref = s.measure_1q(range(n), "Z")
        sites, dims = _device_state(torch, s, batch, n, cap)
    bad_dims = dims.clone()
    bad_dims[1, 1] = cap + 1          # instance 1: a bond dimension above chi_cap
    bad_dims[2, n] = 5                # instance 2: the right edge must be 1
    qubits = torch.tensor(list(range(n - 1)) + [n], device="cuda", dtype=torch.int32)   # last one out of range
    got = _call(lib, torch, sites, bad_dims, n, batch, cap, qubits, "Z")
    assert np.all(np.isnan(got[1])) and np.all(np.isnan(got[2]))
    assert np.all(np.isnan(got[:, n - 1]))
    assert np.abs(got[0, :n - 1] - ref[0, :n - 1]).max() <= TOL
    good = _call(lib, torch, sites, dims, n, batch, cap, torch.arange(n, device="cuda", dtype=torch.int32), "Z")
    assert np.abs(good - ref).max() <= TOL


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
