"""The adjoint at the gradient workload's geometry: N = 24 ring (closing bond
through swap gates, 91 ops per step), chi_max = 64, cutoff 1e-10, dt = 0.05,
under a seeded model with every term switched on, from a generic entangled
state at chi = 64 (the product state evolved ten steps of 0.3 by the same
model; its Schmidt spectra have no degeneracy at the cut, so the truncation
with the ranks held fixed is a smooth map, and the 64th Schmidt value is ~4e-4
of the largest: the truncated-SVD backward divides by the kept s_j^2, and after
four steps, with s_64 ~ 5e-6 s_0, the SVD's rounding amplified by 1/s^2 moved
the directional derivatives by 0.5%); loss = sum_{i<j} connected
<Z_i Z_j> after two steps.  Random directional derivatives of the gradient
against central finite differences of the forward run with its ranks held
fixed, FP64 and mixed contractions.  The step is h = 1e-4: the directional
derivatives are ~5e-4 while the loss carries ~1e-12 of rounding from the SVDs,
so at h = 1e-6 the difference quotient itself is noisy at 1e-6 (measured: two
precisions' quotients differ by 6e-7); at 1e-4 rounding contributes ~1e-8
and the truncation error (h^2 times the third derivative) stays below that."""
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


def _moved(wl, v, h):
    w = W.Workload(**{f: (np.array(x, copy=True) if isinstance(x, np.ndarray) else x) for f, x in wl.__dict__.items()})
    n, nb = w.n, len(w.bonds)
    for k, name in enumerate(["h_x", "h_y", "h_z", "g0", "g1", "g2"]):
        getattr(w, name)[0] += h * v[k * n:(k + 1) * n]
    w.J[0] += h * v[6 * n:6 * n + nb]
    w.Jz[0] += h * v[6 * n + nb:]
    return w


@pytest.mark.parametrize("precision", ["tf32", "fp64"])
def test_ring24_directional_derivatives(precision):
    from paper_2203_05871_gb300 import FP64, MIXED_TF32, Solver
    wl = W.random_model(24, W.ring_bonds(24), 2203058714, chi_max=64, cutoff=1e-10, dt=0.05, steps=2)
    n, nb, steps = 24, len(wl.bonds), 2
    with Solver(n, batch=1, chi_cap=64) as w:
        w.build_gates(wl, dt=0.3)
        w.step(10)
        dims, tens = w.get_state(0)
    zb = np.zeros((1, n))
    wb = np.triu(np.ones((1, n, n)), 1)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    # an explicit strict Jacobi tolerance: the finite differences divide the
    # difference of two forward runs by 2h, so their SVDs must be converged to
    # rounding (the mixed path's default finish tolerance is 1e-10)
    s = Solver(n, batch=1, chi_cap=64, precision=FP64 if precision == "fp64" else MIXED_TF32, jacobi_tol=1e-14)

    def start(w):
        s.build_gates(w)
        s.set_state(0, dims, tens)

    start(wl)
    s.grad_forward(steps)
    ranks = s.rank_log(steps)
    g, L = s.grad_backward(zb, wb)
    assert int(s.status()["chi"].max()) == 64

    def loss(w):
        start(w)
        s.force_ranks(ranks)
        s.step(steps)
        s.force_ranks(None)
        return float(s.measure_2q(pairs, "ZZ", connected=True)[0].sum())

    assert abs(loss(wl) - L[0]) <= 1e-9 * max(1.0, abs(L[0]))
    rng = np.random.default_rng(24)
    h = 1e-4
    for trial in range(2):
        v = np.zeros(6 * n + 2 * nb)
        for k in (0, 2, 3, 5):                      # h_x, h_z, g0, g2 per qubit
            v[k * n:(k + 1) * n] = rng.normal(size=n)
        v[6 * n:6 * n + nb] = rng.normal(size=nb)   # J per bond
        v /= np.linalg.norm(v)
        fd = (loss(_moved(wl, v, h)) - loss(_moved(wl, v, -h))) / (2 * h)
        ad = float(g[0] @ v)
        print(f"ring24 chi64 {precision}: direction {trial}: adjoint {ad:.10e}, finite difference {fd:.10e}, "
              f"|d| = {abs(ad - fd):.2e}")
        assert abs(ad - fd) <= 1e-8 + 1e-4 * abs(fd)
