"""CPU tests of the C-ABI library: it loads, exports every symbol that
include/mpdo.h declares, and its host-only scheduler reproduces the oracle's
op list.  No compute call needs a GPU here."""
import ctypes
import os
import re

import pytest

import workloads as W
from oracle import schedule

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_05871_gb300 import build as B
    B.build()
    from paper_2203_05871_gb300 import mpdo
    return mpdo.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mpdo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpdo_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for need in ("mpdo_init", "mpdo_build_gates", "mpdo_trotter_step", "mpdo_measure_1q", "mpdo_measure_2q",
                 "mpdo_status", "mpdo_last_error", "mpdo_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2203_05871_gb300 import mpdo
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(mpdo.exported_symbols()) == declared_symbols()


@pytest.mark.parametrize("n,bonds", [(8, W.chain_bonds(8)), (24, W.ring_bonds(24)), (5, W.ring_bonds(5)),
                                     (40, W.grid_snake_bonds(10, 4)), (12, W.grid_snake_bonds(4, 3)),
                                     (6, [(0, 5), (1, 2), (3, 4), (2, 4), (0, 1)])])
def test_library_schedule_equals_oracle(lib, n, bonds):
    from paper_2203_05871_gb300 import mpdo
    ref = [[tuple(o) for o in L] for L in schedule.step_layers(n, bonds)]
    assert mpdo.schedule(n, bonds) == ref


def test_schedule_rejects_bad_graphs(lib):
    from paper_2203_05871_gb300 import mpdo
    for n, bonds in [(4, [(0, 1), (1, 2)]),          # qubit 3 has no bond
                     (3, [(0, 0), (1, 2)]),          # self bond
                     (3, [(0, 1), (1, 0), (1, 2)]),  # duplicate
                     (3, [(0, 3), (1, 2)])]:         # out of range
        with pytest.raises(mpdo.MpdoError) as e:
            mpdo.schedule(n, bonds)
        assert e.value.code == mpdo.MPDO_EINVAL
    assert lib.mpdo_last_error().decode() != ""


def test_init_rejects_bad_config_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_2203_05871_gb300 import mpdo
    cfg = mpdo.Config()
    assert lib.mpdo_config_default(ctypes.byref(cfg)) == 0
    h = ctypes.c_void_p()
    cfg.n_qubits, cfg.batch, cfg.chi_cap = 2, 1, 8
    assert lib.mpdo_init(ctypes.byref(h), ctypes.byref(cfg), None) == mpdo.MPDO_EINVAL
    cfg.n_qubits, cfg.chi_cap = 8, 1024
    assert lib.mpdo_init(ctypes.byref(h), ctypes.byref(cfg), None) == mpdo.MPDO_EINVAL
    cfg.chi_cap, cfg.trotter_order = 16, 3
    assert lib.mpdo_init(ctypes.byref(h), ctypes.byref(cfg), None) == mpdo.MPDO_EINVAL
    cfg.trotter_order = 2
    for bad in (2.0, float("nan")):
        cfg.precond_rho = bad
        assert lib.mpdo_init(ctypes.byref(h), ctypes.byref(cfg), None) == mpdo.MPDO_EINVAL
        assert "precond_rho" in lib.mpdo_last_error().decode()
