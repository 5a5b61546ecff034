"""Failure detection without a GPU fault.

Every device-side wait is bounded and every per-instance failure is a status
bit, so a bad instance cannot stop the step or corrupt the other instances:
  - a Jacobi sweep limit that is too small returns ENOCONV, and mpdo_status
    flags only the instance whose SVDs did not converge;
  - a cooperative barrier whose CTA never arrives (a CTA left out of the QR
    launch on the host, mpdo_inject_fault) gives up after barrier_timeout_ms:
    the kernel returns, the step returns ETIMEOUT, and the GPU stays usable;
  - a non-finite tensor loaded into one instance returns ENONFINITE for that
    instance only, and the other instances evolve bit for bit as in a clean
    batched run."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import build as B
    B.build()


def _identity_model(wl, b):
    """All parameters of instance b set to zero: every gate is the identity."""
    for name in ("h_x", "h_y", "h_z", "g0", "g1", "g2"):
        getattr(wl, name)[b, :] = 0.0
    wl.J[b, :] = 0.0
    wl.Jz[b, :] = 0.0


def test_sweep_limit_flags_only_the_unconverged_instance():
    """jacobi_max_sweeps = 1.  Instance 0 holds the (unnormalised) maximally
    mixed product state (every site vector e_I) under identity gates: each bond
    matrix has a single non-zero entry, its QR is exact and the Jacobi pass
    meets no pair to rotate.  Instance 1 is an entangled random state under a
    random model, whose SVDs need several sweeps."""
    from paper_2203_05871_gb300 import MPDO_ENOCONV, ST_NOCONV, Solver
    n = 8
    wl = W.random_model(n, W.chain_bonds(n), 301, batch=2, chi_max=16, cutoff=1e-12)
    _identity_model(wl, 0)
    s = Solver(n, batch=2, chi_cap=16, jacobi_max_sweeps=1)
    s.build_gates(wl)
    dims0 = [1] * (n + 1)
    s.set_state(0, dims0, [np.array([1.0, 0.0, 0.0, 0.0]).reshape(1, 4, 1) for _ in range(n)])
    dims1, tens1 = W.random_mpo_state(n, 16, seed=302)
    s.set_state(1, dims1, tens1)
    rc = s.step(2, check=False)
    assert rc == MPDO_ENOCONV
    st = s.status()
    assert st["status"][0] == 0
    assert st["status"][1] & ST_NOCONV
    # the step still ran to the end: the unconverged instance is finite, the other exact
    z = s.measure_1q(range(n), "Z")
    assert np.all(np.isfinite(z))
    assert np.all(z[0] == 0.0)
    s.close()


def test_barrier_timeout_returns_and_context_stays_usable():
    """One CTA of a QR op is left out of the launch on the host; the op's other
    CTAs wait for it at their first barrier, give up after 1 ms, record
    ST_TIMEOUT and return.  The step returns ETIMEOUT instead of hanging, and
    a fresh context on the same GPU then runs clean."""
    from paper_2203_05871_gb300 import MPDO_ETIMEOUT, ST_TIMEOUT, Solver
    n, chi = 8, 64
    wl = W.random_model(n, W.chain_bonds(n), 303, chi_max=chi, cutoff=1e-12)
    dims, tens = W.random_mpo_state(n, chi, seed=304)
    s = Solver(n, batch=1, chi_cap=chi, barrier_timeout_ms=1)
    s.build_gates(wl)
    s.set_state(0, dims, tens)
    s.inject_fault()
    rc = s.step(1, check=False)
    assert rc == MPDO_ETIMEOUT
    assert s.status()["status"][0] & ST_TIMEOUT
    s.close()
    f = Solver(n, batch=1, chi_cap=chi)
    f.build_gates(wl)
    f.set_state(0, dims, tens)
    assert f.step(1, check=False) == 0
    assert f.status()["status"][0] == 0
    assert np.all(np.isfinite(f.measure_1q(range(n), "Z")))
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_instance_is_isolated(precision):
    """A NaN entry in instance 1 of 3: the step returns ENONFINITE, only
    instance 1 carries ST_NONFINITE, and instances 0 and 2 equal, bit for bit,
    the same instances of a batched run where instance 1 is clean."""
    from paper_2203_05871_gb300 import FP64, MIXED_TF32, MPDO_ENONFINITE, ST_NONFINITE, Solver
    prec = FP64 if precision == "fp64" else MIXED_TF32
    n, chi, steps = 8, 32, 3
    wl = W.random_model(n, W.chain_bonds(n), 305, batch=3, chi_max=chi, cutoff=1e-12)
    states = [W.random_mpo_state(n, chi, seed=306 + b) for b in range(3)]

    def run(poison):
        s = Solver(n, batch=3, chi_cap=chi, precision=prec)
        s.build_gates(wl)
        for b, (d, t) in enumerate(states):
            t = [x.copy() for x in t]
            if poison and b == 1:
                t[3][0, 1, 0] = np.nan
            s.set_state(b, d, t)
        rc = s.step(steps, check=False)
        out = (rc, s.status()["status"].copy(), [s.get_state(b) for b in range(3)])
        s.close()
        return out

    rc_bad, st_bad, st8_bad = run(True)
    rc_ok, st_ok, st8_ok = run(False)
    assert rc_ok == 0 and np.all(st_ok == 0)
    assert rc_bad == MPDO_ENONFINITE
    assert st_bad[1] & ST_NONFINITE
    assert st_bad[0] == 0 and st_bad[2] == 0
    for b in (0, 2):
        (da, ta), (db, tb) = st8_bad[b], st8_ok[b]
        assert da == db
        for x, y in zip(ta, tb):
            assert np.array_equal(x, y)
