"""Test-side conversions between the oracle's real form and the library's storage."""
import numpy as np

from oracle import csvd


def q_storage(U):
    """Rows [Re Q | Im Q] of the complex N x n form of a 2N x 2n block matrix U."""
    N, n = U.shape[0] // 2, U.shape[1] // 2
    return np.ascontiguousarray(np.hstack([U[:N, :n], U[N:, :n]]))


def U_of(Qs):
    n = Qs.shape[1] // 2
    return csvd.U_from_Q(Qs[:, :n] + 1j * Qs[:, n:])


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
