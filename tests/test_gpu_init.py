"""Device truncated complex SVD start (vp_init_csvd, Sec. 3.2 / Algorithm 2)
against the oracle and the properties that fix it."""
import numpy as np
import pytest

import workloads as W
from oracle import csvd
from tests.helpers import U_of, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_05555_gb300 import Context
    return Context(0)


def T(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


@pytest.mark.parametrize("N,p,n,quiet", [(3001, 37, 5, False), (20_000, 64, 10, False),
                                         (4000, 16, 3, True), (501, 7, 7, False),
                                         (3000, 256, 16, False), (2000, 200, 40, False)])
def test_init_csvd(ctx, N, p, n, quiet):
    etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    X0, V0 = W.load_batch(W.TWO_STREAM, etas, N, quiet=quiet)
    Q, Z, sig = ctx.init_csvd(T(X0), T(V0), n)
    ctx.sync_status()
    Qg, Zg, sg = Q.cpu().numpy(), Z.cpu().numpy(), sig.cpu().numpy()
    Rc = (X0 + 1j * V0).T
    s_ref = np.linalg.svd(Rc, compute_uv=False)
    assert rel(sg[:n], s_ref[:n]) < 1e-10
    U = U_of(Qg)
    R0 = np.vstack([X0.T, V0.T])
    # Eckart-Young: the residual of the n-term projection is the tail of the
    # spectrum (eigenvalues of R^H R from an independent CPU routine)
    ev = np.sort(np.linalg.eigvalsh(Rc.conj().T @ Rc))[::-1]
    np.testing.assert_allclose(np.linalg.norm(R0 - U @ Zg) ** 2, ev[n:].sum(),
                               rtol=1e-8, atol=1e-12 * ev.sum())
    Qc = Qg[:, :n] + 1j * Qg[:, n:]
    assert np.linalg.norm(Qc.conj().T @ Qc - np.eye(n)) < 1e-12
    # zeta = Q^H R0
    assert rel(Zg, np.vstack([(Qc.conj().T @ Rc).real, (Qc.conj().T @ Rc).imag])) < 1e-12
    if quiet:
        # well separated spectrum: the subspace, hence U Z, is unique
        Uo, Zo, _ = csvd.csvd_init(X0, V0, n)
        assert rel(U @ Zg, Uo @ Zo) < 1e-10


@pytest.mark.parametrize("family,quiet,n_min,n_max,tol", [
    (W.TWO_STREAM, True, 1, 10, 1e-8), (W.LANDAU, True, 2, 12, 1e-12),
    (W.BUMP_ON_TAIL, False, 3, 8, 1e-3), (W.BUMP_ON_TAIL, True, 8, 16, 1e-30)])
def test_init_csvd_rank(ctx, family, quiet, n_min, n_max, tol):
    """Rank chosen from the singular values: the smallest n in [n_min, n_max]
    with relative tail energy < tol, lowered while sigma_n < 1e-6 sigma_1;
    the state equals the fixed-rank start with that n, bit for bit."""
    N, p = 4000, 16
    if family is W.LANDAU:
        etas = [{"alpha": a, "sigma": 1.0} for a in np.linspace(0.01, 0.05, p)]
    elif family is W.TWO_STREAM:
        etas = W.hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    else:
        etas = W.hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})
    X0, V0 = W.load_batch(family, etas, N, quiet=quiet)
    Q, Z, sig, n = ctx.init_csvd_rank(T(X0), T(V0), n_min, n_max, tol)
    ctx.sync_status()
    s = np.linalg.svd((X0 + 1j * V0).T, compute_uv=False)
    e = s ** 2
    tail = 1.0 - np.cumsum(e) / e.sum()
    want = next((k + 1 for k in range(n_min - 1, n_max) if tail[k] < tol), n_max)
    while s[want - 1] < 1e-6 * s[0]:
        want -= 1
    assert n == want
    Qf, Zf, _ = ctx.init_csvd(T(X0), T(V0), n)
    assert torch.equal(Q, Qf) and torch.equal(Z, Zf)
