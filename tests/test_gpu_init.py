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
                                         (4000, 16, 3, True), (501, 7, 7, False)])
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
