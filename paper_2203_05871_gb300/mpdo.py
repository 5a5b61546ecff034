"""Thin ctypes binding of libmpdo (include/mpdo.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; this module only
converts numpy / torch arguments to pointers.  If the shared library is
missing it raises immediately: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmpdo.so")

MPDO_OK, MPDO_EINVAL, MPDO_ENOMEM, MPDO_ECUDA, MPDO_ENOCONV, MPDO_ETIMEOUT, MPDO_ENONFINITE, \
    MPDO_ECAPACITY, MPDO_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
ST_NOCONV, ST_NONFINITE, ST_TIMEOUT, ST_CAPACITY = 1, 2, 4, 8
FP64, MIXED_TF32, MIXED_BF16X3 = 0, 1, 2
FAULT_DROP_CTA = 1
STORE_F64, STORE_F32 = 0, 1

_ERR_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOCONV", -5: "ETIMEOUT",
              -6: "ENONFINITE", -7: "ECAPACITY", -8: "ESTATE"}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class Config(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("batch", ctypes.c_int), ("chi_cap", ctypes.c_int),
                ("precision", ctypes.c_int), ("storage", ctypes.c_int), ("trotter_order", ctypes.c_int),
                ("force_trace", ctypes.c_int), ("jacobi_max_sweeps", ctypes.c_int),
                ("jacobi_tol", ctypes.c_double), ("barrier_timeout_ms", ctypes.c_uint),
                ("max_slots", ctypes.c_int), ("device", ctypes.c_int), ("qr_blocked", ctypes.c_int),
                ("precond_rho", ctypes.c_double)]


class Model(ctypes.Structure):
    _fields_ = [("h_x", _dp), ("h_y", _dp), ("h_z", _dp), ("g0", _dp), ("g1", _dp), ("g2", _dp),
                ("n_bonds", ctypes.c_int), ("bond_i", _ip), ("bond_j", _ip), ("J", _dp), ("Jz", _dp),
                ("chi_max", _ip), ("cutoff", _dp), ("init_pauli", ctypes.c_char_p)]


class MpdoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmpdo {_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmpdo.so (built by paper_2203_05871_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmpdo is not built ({path} missing); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    sig = {
        "mpdo_config_default": (ctypes.c_int, [ctypes.POINTER(Config)]),
        "mpdo_init": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(Config), vp]),
        "mpdo_build_gates": (ctypes.c_int, [vp, ctypes.POINTER(Model), ctypes.c_double]),
        "mpdo_trotter_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "mpdo_trotter_step_graph": (ctypes.c_int, [vp, ctypes.c_int]),
        "mpdo_measure_1q": (ctypes.c_int, [vp, _ip, ctypes.c_int, ctypes.c_char, vp, ctypes.c_int]),
        "mpdo_measure_2q": (ctypes.c_int, [vp, _ip, ctypes.c_int, ctypes.c_char_p, ctypes.c_int, vp,
                                           ctypes.c_int]),
        "mpdo_status": (ctypes.c_int, [vp, _ip, _dp, _ip, _dp]),
        "mpdo_set_state": (ctypes.c_int, [vp, ctypes.c_int, _ip, _dp]),
        "mpdo_get_state": (ctypes.c_int, [vp, ctypes.c_int, _ip, _dp, ctypes.c_longlong]),
        "mpdo_op_counts": (ctypes.c_int, [vp, _ip, _ip, _ip]),
        "mpdo_rank_log": (ctypes.c_int, [vp, _ip, ctypes.c_longlong]),
        "mpdo_gates": (ctypes.c_int, [vp, ctypes.c_int, _dp, ctypes.c_longlong]),
        "mpdo_schedule": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _ip, _ip, _ip, ctypes.c_longlong, _ip]),
        "mpdo_profile_enable": (ctypes.c_int, [vp, ctypes.c_int]),
        "mpdo_profile_read": (ctypes.c_int, [vp, _dp, ctypes.POINTER(ctypes.c_longlong), _dp, ctypes.c_int,
                                             ctypes.c_int]),
        "mpdo_profile_sweeps": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_longlong),
                                               ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "mpdo_profile_sweeps_critical": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_longlong),
                                                        ctypes.POINTER(ctypes.c_longlong),
                                                        ctypes.POINTER(ctypes.c_longlong)]),
        "mpdo_measure_1q_noalloc": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                                   ctypes.c_int, ctypes.c_char, vp, vp]),
        "mpdo_force_ranks": (ctypes.c_int, [vp, _ip, ctypes.c_int]),
        "mpdo_inject_fault": (ctypes.c_int, [vp, ctypes.c_int]),
        "mpdo_renyi2": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "mpdo_init_graph_state": (ctypes.c_int, [vp, _ip, ctypes.c_int]),
        "mpdo_gemm_tc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int,
                                        vp, ctypes.c_int, ctypes.c_int, vp]),
        "mpdo_osee": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
        "mpdo_autotune": (ctypes.c_int, [vp, _ip, ctypes.c_int, _ip]),
        "mpdo_grad_forward": (ctypes.c_int, [vp, ctypes.c_int]),
        "mpdo_grad_backward": (ctypes.c_int, [vp, _dp, _dp, _dp, _dp]),
        "mpdo_grad": (ctypes.c_int, [vp, ctypes.c_int, _dp, _dp, _dp, _dp]),
        "mpdo_last_error": (ctypes.c_char_p, []),
        "mpdo_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    """Names declared in include/mpdo.h (for the export test)."""
    return ["mpdo_config_default", "mpdo_init", "mpdo_build_gates", "mpdo_trotter_step", "mpdo_trotter_step_graph",
            "mpdo_measure_1q",
            "mpdo_measure_2q", "mpdo_status", "mpdo_set_state", "mpdo_get_state", "mpdo_op_counts",
            "mpdo_rank_log", "mpdo_force_ranks", "mpdo_autotune", "mpdo_gates", "mpdo_schedule", "mpdo_profile_enable",
            "mpdo_profile_read", "mpdo_profile_sweeps", "mpdo_profile_sweeps_critical", "mpdo_measure_1q_noalloc", "mpdo_inject_fault", "mpdo_renyi2", "mpdo_osee", "mpdo_gemm_tc", "mpdo_init_graph_state", "mpdo_grad_forward",
            "mpdo_grad_backward", "mpdo_grad", "mpdo_last_error", "mpdo_destroy"]


PROFILE_KINDS = ["merge_gate", "jacobi_svd", "truncate", "reconstruct", "trace", "measure", "build_gates",
                 "jacobi_fp32", "precond_gemm", "qr"]


def schedule(n: int, bonds):
    """Host-only op list of one Trotter step: list of layers of
    (kind, p, qa, qb, bond, frac) tuples, as computed by libmpdo."""
    lib = load_library()
    bi = _as([b[0] for b in bonds], np.int32)
    bj = _as([b[1] for b in bonds], np.int32)
    cnt = ctypes.c_int()
    _check(lib.mpdo_schedule(n, len(bonds), _ptr(bi, ctypes.c_int), _ptr(bj, ctypes.c_int), None, 0,
                             ctypes.byref(cnt)))
    buf = np.zeros(cnt.value * 7, np.int32)
    _check(lib.mpdo_schedule(n, len(bonds), _ptr(bi, ctypes.c_int), _ptr(bj, ctypes.c_int),
                             _ptr(buf, ctypes.c_int), len(buf), ctypes.byref(cnt)))
    layers = []
    for r in buf.reshape(-1, 7):
        li, kind, p, qa, qb, bond, f2 = (int(x) for x in r)
        while len(layers) <= li:
            layers.append([])
        layers[li].append(("swap" if kind else "gate", p, qa, qb, bond, f2 / 2.0))
    return layers


def gemm_tc(A, B, kind: int = MIXED_TF32, stream=None):
    """C = A B (CUDA float64 torch tensors, row-major) by the library's
    FP64-accurate tensor-core GEMM (mpdo_gemm_tc); returns C."""
    import torch
    lib = load_library()
    M, K = A.shape
    K2, N = B.shape
    assert K == K2 and A.dtype == torch.float64 and B.dtype == torch.float64
    A, B = A.contiguous(), B.contiguous()
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    st = ctypes.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    _check(lib.mpdo_gemm_tc(M, N, K, ctypes.c_void_p(A.data_ptr()), K, ctypes.c_void_p(B.data_ptr()), N,
                            ctypes.c_void_p(C.data_ptr()), N, int(kind), st))
    return C


def _check(code):
    if code != MPDO_OK:
        raise MpdoError(code, _lib.mpdo_last_error().decode())
    return code


def _as(arr, dtype):
    return np.ascontiguousarray(np.asarray(arr, dtype=dtype))


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Solver:
    """One libmpdo context: B instances of an N-qubit model on one GPU.

    The keyword arguments fill ``mpdo_config`` (include/mpdo.h documents each
    field): ``precision`` FP64, MIXED_TF32 or MIXED_BF16X3; ``storage``
    STORE_F64 or STORE_F32; ``trotter_order`` 2 or 4; ``jacobi_tol`` and
    ``jacobi_max_sweeps`` of the SVD; ``barrier_timeout_ms`` bounding every
    device-side wait; ``max_slots`` (ops in flight, 0 = automatic);
    ``qr_blocked`` (mixed path: the blocked QR instead of the column QR);
    ``precond_rho`` (mixed path: the FP32 preconditioning sweeps' stop
    threshold, 0 = 1e-3); ``stream`` a torch stream or a raw cudaStream_t.
    """

    def __init__(self, n_qubits: int, batch: int = 1, chi_cap: int = 32, precision: int = FP64,
                 storage: int = STORE_F64, stream=None, force_trace: bool = True, jacobi_max_sweeps: int = 100,
                 jacobi_tol: float = 0.0, barrier_timeout_ms: int = 4000, max_slots: int = 0,
                 device: Optional[int] = None, trotter_order: int = 2, qr_blocked: bool = False,
                 precond_rho: float = 0.0):
        lib = load_library()
        cfg = Config()
        _check(lib.mpdo_config_default(ctypes.byref(cfg)))
        cfg.n_qubits, cfg.batch, cfg.chi_cap = n_qubits, batch, chi_cap
        cfg.precision, cfg.storage = precision, storage
        cfg.force_trace = 1 if force_trace else 0
        cfg.jacobi_max_sweeps, cfg.jacobi_tol = jacobi_max_sweeps, jacobi_tol
        cfg.barrier_timeout_ms, cfg.max_slots = barrier_timeout_ms, max_slots
        cfg.trotter_order = int(trotter_order)
        cfg.qr_blocked = 1 if qr_blocked else 0
        cfg.precond_rho = float(precond_rho)
        if device is None:
            try:
                import torch
                device = torch.cuda.current_device() if torch.cuda.is_available() else -1
            except Exception:
                device = -1
        cfg.device = int(device)
        self._lib = lib
        self.n, self.batch, self.chi_cap = n_qubits, batch, chi_cap
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None
                                                                     else None))
        _check(lib.mpdo_init(ctypes.byref(h), ctypes.byref(cfg), st))
        self._h = h
        self._keep = []

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mpdo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- model -----------------------------------------------------------
    def build_gates(self, wl, dt: Optional[float] = None):
        """wl: a workloads.Workload with batch == self.batch."""
        B, N = self.batch, self.n
        assert wl.batch == B and wl.n == N
        arrs = dict(h_x=_as(wl.h_x, np.float64), h_y=_as(wl.h_y, np.float64), h_z=_as(wl.h_z, np.float64),
                    g0=_as(wl.g0, np.float64), g1=_as(wl.g1, np.float64), g2=_as(wl.g2, np.float64),
                    J=_as(wl.J, np.float64), Jz=_as(wl.Jz, np.float64))
        bi = _as([b[0] for b in wl.bonds], np.int32)
        bj = _as([b[1] for b in wl.bonds], np.int32)
        chi = _as(wl.chi_max, np.int32)
        cut = _as(wl.cutoff, np.float64)
        m = Model()
        for k, a in arrs.items():
            setattr(m, k, _ptr(a, ctypes.c_double))
        m.n_bonds = len(wl.bonds)
        m.bond_i, m.bond_j = _ptr(bi, ctypes.c_int), _ptr(bj, ctypes.c_int)
        m.chi_max, m.cutoff = _ptr(chi, ctypes.c_int), _ptr(cut, ctypes.c_double)
        init = None
        if wl.init is not None:
            init = "".join(s.lower() for s in wl.init).encode()
        m.init_pauli = init
        _check(self._lib.mpdo_build_gates(self._h, ctypes.byref(m), float(wl.dt if dt is None else dt)))
        self._n_bonds = len(wl.bonds)

    def init_graph_state(self, pairs):
        """Graph state of Sec. 2.2: +x everywhere, then CZ on every pair."""
        p = _as(pairs, np.int32).reshape(-1, 2)
        _check(self._lib.mpdo_init_graph_state(self._h, _ptr(p, ctypes.c_int) if len(p) else None, len(p)))

    def step(self, n_steps: int = 1, check: bool = True, graph: bool = False):
        """n_steps Trotter steps (graph=True: replay the step captured as a CUDA graph)."""
        fn = self._lib.mpdo_trotter_step_graph if graph else self._lib.mpdo_trotter_step
        rc = fn(self._h, int(n_steps))
        if check:
            _check(rc)
        return rc

    # -- observables -----------------------------------------------------
    def measure_1q(self, qubits: Sequence[int], comp: str = "Z", out=None):
        """[B, nq] numpy array, or fills ``out`` (a CUDA torch tensor) in place."""
        q = _as(qubits, np.int32)
        if out is not None:
            _check(self._lib.mpdo_measure_1q(self._h, _ptr(q, ctypes.c_int), len(q), comp.encode(),
                                             ctypes.c_void_p(out.data_ptr()), 1))
            return out
        res = np.zeros((self.batch, len(q)))
        _check(self._lib.mpdo_measure_1q(self._h, _ptr(q, ctypes.c_int), len(q), comp.encode(),
                                         res.ctypes.data_as(ctypes.c_void_p), 0))
        return res

    def measure_2q(self, pairs, comps: str = "ZZ", connected: bool = True, out=None):
        p = _as(pairs, np.int32).reshape(-1, 2)
        if out is not None:
            _check(self._lib.mpdo_measure_2q(self._h, _ptr(p, ctypes.c_int), len(p), comps.encode(),
                                             int(connected), ctypes.c_void_p(out.data_ptr()), 1))
            return out
        res = np.zeros((self.batch, len(p)))
        _check(self._lib.mpdo_measure_2q(self._h, _ptr(p, ctypes.c_int), len(p), comps.encode(), int(connected),
                                         res.ctypes.data_as(ctypes.c_void_p), 0))
        return res

    def renyi2(self):
        """Second Renyi entropy S2 = -ln tr(rho^2) of every instance, [B]."""
        res = np.zeros(self.batch)
        _check(self._lib.mpdo_renyi2(self._h, res.ctypes.data_as(ctypes.c_void_p), 0))
        return res

    def osee(self, bond: Optional[int] = None):
        """Operator space entanglement entropy at the cut after path position
        ``bond`` (default: the central bond N/2 - 1), [B]."""
        if bond is None:
            bond = self.n // 2 - 1
        res = np.zeros(self.batch)
        _check(self._lib.mpdo_osee(self._h, int(bond), res.ctypes.data_as(ctypes.c_void_p), 0))
        return res

    # -- state and diagnostics ------------------------------------------
    def status(self):
        B, N = self.batch, self.n
        st = np.zeros(B, np.int32)
        md = np.zeros(B)
        chi = np.zeros((B, N - 1), np.int32)
        tr = np.zeros(B)
        _check(self._lib.mpdo_status(self._h, _ptr(st, ctypes.c_int), _ptr(md, ctypes.c_double),
                                     _ptr(chi, ctypes.c_int), _ptr(tr, ctypes.c_double)))
        return {"status": st, "max_discarded": md, "chi": chi, "trace_before": tr}

    def set_state(self, b: int, dims, tensors):
        d = _as(dims, np.int32)
        flat = np.concatenate([np.asarray(t, np.float64).reshape(-1) for t in tensors])
        _check(self._lib.mpdo_set_state(self._h, int(b), _ptr(d, ctypes.c_int), _ptr(flat, ctypes.c_double)))

    def get_state(self, b: int = 0):
        d = np.zeros(self.n + 1, np.int32)
        _check(self._lib.mpdo_get_state(self._h, int(b), _ptr(d, ctypes.c_int), None, 0))
        tot = int(sum(int(d[p]) * 4 * int(d[p + 1]) for p in range(self.n)))
        buf = np.zeros(max(tot, 1))
        _check(self._lib.mpdo_get_state(self._h, int(b), _ptr(d, ctypes.c_int), _ptr(buf, ctypes.c_double), tot))
        out, off = [], 0
        for p in range(self.n):
            sz = int(d[p]) * 4 * int(d[p + 1])
            out.append(buf[off:off + sz].reshape(int(d[p]), 4, int(d[p + 1])).copy())
            off += sz
        return [int(x) for x in d], out

    def op_counts(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.mpdo_op_counts(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def gates(self, b: int = 0):
        n_ops = self.op_counts()[0]
        buf = np.zeros(n_ops * 256)
        _check(self._lib.mpdo_gates(self._h, int(b), _ptr(buf, ctypes.c_double), len(buf)))
        return buf.reshape(n_ops, 16, 16)

    def profile(self, on: bool = True):
        _check(self._lib.mpdo_profile_enable(self._h, int(on)))

    def profile_read(self, reset: bool = False):
        sw, sv, s32 = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._lib.mpdo_profile_sweeps(self._h, ctypes.byref(sw), ctypes.byref(sv), ctypes.byref(s32)))
        cr, cr32, nch = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._lib.mpdo_profile_sweeps_critical(self._h, ctypes.byref(cr), ctypes.byref(cr32),
                                                      ctypes.byref(nch)))
        K = len(PROFILE_KINDS)
        ms = np.zeros(K)
        ln = np.zeros(K, np.int64)
        fl = np.zeros(K)
        _check(self._lib.mpdo_profile_read(self._h, _ptr(ms, ctypes.c_double), ln.ctypes.data_as(
            ctypes.POINTER(ctypes.c_longlong)), _ptr(fl, ctypes.c_double), K, int(reset)))
        out = {k: {"ms": float(ms[i]), "launches": int(ln[i]), "flops": float(fl[i])}
               for i, k in enumerate(PROFILE_KINDS)}
        out["jacobi_svd"]["sweeps"] = int(sw.value)
        out["jacobi_svd"]["svds"] = int(sv.value)
        out["jacobi_svd"]["sweeps_fp32"] = int(s32.value)
        out["jacobi_svd"]["critical_sweeps"] = int(cr.value)
        out["jacobi_svd"]["critical_sweeps_fp32"] = int(cr32.value)
        out["jacobi_svd"]["chunks"] = int(nch.value)
        return out

    def rank_log(self, n_steps: int):
        n_ops = self.op_counts()[0]
        buf = np.zeros(self.batch * n_steps * n_ops, np.int32)
        _check(self._lib.mpdo_rank_log(self._h, _ptr(buf, ctypes.c_int), len(buf)))
        return buf.reshape(self.batch, n_steps * n_ops)

    def force_ranks(self, ranks=None):
        """Hold the truncation ranks of the next steps fixed: ranks is
        [B, n_steps * n_ops] (the layout of rank_log); None clears."""
        if ranks is None:
            _check(self._lib.mpdo_force_ranks(self._h, None, 0))
            return
        n_ops = self.op_counts()[0]
        r = _as(ranks, np.int32).reshape(self.batch, -1)
        assert r.shape[1] % n_ops == 0
        _check(self._lib.mpdo_force_ranks(self._h, _ptr(r, ctypes.c_int), r.shape[1] // n_ops))

    def inject_fault(self, kind: int = FAULT_DROP_CTA):
        """Host-side fault injection (mpdo_inject_fault): the next QR launch
        leaves out one CTA of an op, whose barrier then times out."""
        _check(self._lib.mpdo_inject_fault(self._h, int(kind)))

    # -- adjoint ----------------------------------------------------------
    def n_params(self):
        return 6 * self.n + 2 * self._n_bonds

    def grad_forward(self, n_steps: int):
        """n_steps Trotter steps with per-step checkpoints for grad_backward."""
        _check(self._lib.mpdo_grad_forward(self._h, int(n_steps)))

    def grad_backward(self, zbar=None, wbar=None):
        """Gradient of sum_i zbar[b,i] <z_i> + sum_{i<j} wbar[b,i,j] conn_ij at
        the final time of the last grad_forward.  Returns (grad [B, 6N+2nb],
        loss [B]); grad is packed (h_x, h_y, h_z, g0, g1, g2 per qubit, J, Jz per bond)."""
        B, N = self.batch, self.n
        zb = None if zbar is None else _as(zbar, np.float64).reshape(B, N)
        wb = None if wbar is None else _as(wbar, np.float64).reshape(B, N, N)
        g = np.zeros((B, self.n_params()))
        loss = np.zeros(B)
        _check(self._lib.mpdo_grad_backward(self._h, None if zb is None else _ptr(zb, ctypes.c_double),
                                            None if wb is None else _ptr(wb, ctypes.c_double),
                                            _ptr(g, ctypes.c_double), _ptr(loss, ctypes.c_double)))
        return g, loss

    def autotune(self, classes):
        """Tune the Jacobi block size for each (chi_l, chi_r) in classes; returns
        [n, 2] (FP64 block, FP32 block or 0)."""
        cl = _as(classes, np.int32).reshape(-1, 2)
        out = np.zeros_like(cl)
        _check(self._lib.mpdo_autotune(self._h, _ptr(cl, ctypes.c_int), len(cl), _ptr(out, ctypes.c_int)))
        return out


def saturated_classes(n_qubits: int, chi_max: int):
    """(chi_l, chi_r) of the ops of an n-qubit path once every bond is at its
    largest dimension min(4^(p+1), 4^(n-1-p), chi_max)."""
    d = [1] + [min(4 ** (p + 1), 4 ** (n_qubits - 1 - p), chi_max) for p in range(n_qubits - 1)] + [1]
    return sorted({(d[p], d[p + 2]) for p in range(n_qubits - 1)})
