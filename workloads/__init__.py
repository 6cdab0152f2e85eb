"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the FP64 oracle (``oracle/``) and by the CUDA path
(tests, ``bench.py``).  It holds only input generation: quasi-random (quiet
start) or seeded-random loading of macro-particles from the paper's initial
distributions, parameter sampling, and random ortho-symplectic test matrices.
None of the method's arithmetic (deposit, Poisson, gradients, basis
evolution, initial complex SVD) lives here.

Initial distributions follow Sec. 6.1 (eq. initial_distribution):
f(0,x,v;eta) = f_v(v;eta) * (1 + alpha*cos(k x)) on [0, 2*pi/k) x [-10, 10].
Particles are placed by evaluating the inverse CDF of each factor at the
points of the 2-D Hammersley set of length N (quiet start), or at seeded
uniform random numbers (``quiet=False``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np
from scipy.special import ndtr

BASE_SEED = 20220114
V_MIN, V_MAX = -10.0, 10.0  # velocity domain Omega_v (Sec. 6.1)


# --------------------------------------------------------------------------
# quasi-random points
# --------------------------------------------------------------------------
def radical_inverse_base2(idx: np.ndarray) -> np.ndarray:
    """Van der Corput radical inverse in base 2 of non-negative integers."""
    idx = np.asarray(idx, dtype=np.uint64).copy()
    out = np.zeros(idx.shape, dtype=np.float64)
    scale = 0.5
    while np.any(idx):
        out += (idx & np.uint64(1)).astype(np.float64) * scale
        idx >>= np.uint64(1)
        scale *= 0.5
    return out


def hammersley(N: int) -> tuple[np.ndarray, np.ndarray]:
    """2-D Hammersley set of length N: ((l + 1/2)/N, phi_2(l)), l = 0..N-1."""
    l = np.arange(N, dtype=np.int64)
    return (l + 0.5) / N, radical_inverse_base2(l)


# --------------------------------------------------------------------------
# counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
# "Parallel random numbers: as easy as 1, 2, 3", SC 2011)
# --------------------------------------------------------------------------
_PHILOX_M = (np.uint64(0xD2511F53), np.uint64(0xCD9E8D57))
_PHILOX_W = (np.uint64(0x9E3779B9), np.uint64(0xBB67AE85))
_U32 = np.uint64(0xFFFFFFFF)


def philox4x32(ctr, key, rounds: int = 10):
    """Philox4x32 block: ctr = 4 arrays, key = 2 arrays of 32-bit words (held
    in uint64); returns the 4 output words.  Each round multiplies words 0 and
    2 by the two round constants, mixes the high halves with words 1, 3 and the
    key, and bumps the key by the Weyl constants."""
    c = [np.asarray(x, dtype=np.uint64) & _U32 for x in ctr]
    k0 = np.asarray(key[0], dtype=np.uint64) & _U32
    k1 = np.asarray(key[1], dtype=np.uint64) & _U32
    for _ in range(rounds):
        p0 = _PHILOX_M[0] * c[0]
        p1 = _PHILOX_M[1] * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k0) & _U32, p1 & _U32,
             ((p0 >> np.uint64(32)) ^ c[3] ^ k1) & _U32, p0 & _U32]
        k0 = (k0 + _PHILOX_W[0]) & _U32
        k1 = (k1 + _PHILOX_W[1]) & _U32
    return c


def _u53(a, b):
    """Double in [0, 1) from the top 27 bits of a and 26 bits of b."""
    return ((a >> np.uint64(5)).astype(np.float64) * 67108864.0
            + (b >> np.uint64(6)).astype(np.float64)) * (1.0 / 9007199254740992.0)


def philox_uniforms(N: int, sample: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """(u_x, u_v) of particles l = 0..N-1 of one sample: one Philox4x32-10 block
    per particle with counter (l mod 2^32, l div 2^32, sample, 0) and key
    (seed mod 2^32, seed div 2^32); u_x from words 0-1, u_v from words 2-3."""
    l = np.arange(N, dtype=np.uint64)
    z = np.zeros(N, dtype=np.uint64)
    w = philox4x32([l & _U32, l >> np.uint64(32), z + np.uint64(sample), z],
                   [np.uint64(seed) & _U32, np.uint64(seed) >> np.uint64(32)])
    return _u53(w[0], w[1]), _u53(w[2], w[3])


# --------------------------------------------------------------------------
# inverse CDF sampling (vectorised safeguarded Newton)
# --------------------------------------------------------------------------
def _invert_monotone(cdf: Callable, pdf: Callable, u: np.ndarray, lo: float, hi: float,
                     tol: float = 1e-14, iters: int = 10, table: int = 65537) -> np.ndarray:
    """Solve cdf(x) = u for x in [lo, hi]: a start from a tabulated CDF
    (linear interpolation on `table` points), then bracketed Newton steps
    (a bisection step wherever Newton would leave the bracket)."""
    u = np.asarray(u, dtype=np.float64)
    xs = np.linspace(lo, hi, table)
    cs = cdf(xs)
    x = np.interp(u, cs, xs)
    k = np.clip(np.searchsorted(cs, u), 1, table - 1)
    a, b = xs[k - 1], xs[k]
    for _ in range(iters):
        fx = cdf(x) - u
        a = np.where(fx < 0, x, a)
        b = np.where(fx >= 0, x, b)
        d = pdf(x)
        with np.errstate(divide="ignore", invalid="ignore"):
            xn = x - fx / d
        bad = ~np.isfinite(xn) | (xn < a) | (xn > b)
        xn = np.where(bad, 0.5 * (a + b), xn)
        done = np.abs(xn - x) <= tol * np.maximum(1.0, np.abs(x))
        x = xn
        if np.all(done):
            break
    return x


def sample_positions(u: np.ndarray, alpha: float, k: float) -> np.ndarray:
    """Inverse CDF of f_x(x) = (1 + alpha cos(kx)) / L on [0, L), L = 2 pi / k."""
    L = 2.0 * np.pi / k
    cdf = lambda x: (x + (alpha / k) * np.sin(k * x)) / L
    pdf = lambda x: (1.0 + alpha * np.cos(k * x)) / L
    x = _invert_monotone(cdf, pdf, u, 0.0, L)
    return np.clip(x, 0.0, np.nextafter(L, 0.0))


def _gauss_mixture(weights, means, sigmas):
    w = np.asarray(weights, float) / np.sum(weights)
    m = np.asarray(means, float)
    s = np.asarray(sigmas, float)
    lo_mass = sum(wi * ndtr((V_MIN - mi) / si) for wi, mi, si in zip(w, m, s))
    hi_mass = sum(wi * ndtr((V_MAX - mi) / si) for wi, mi, si in zip(w, m, s))
    Z = hi_mass - lo_mass

    def cdf(v):
        return (sum(wi * ndtr((v - mi) / si) for wi, mi, si in zip(w, m, s)) - lo_mass) / Z

    def pdf(v):
        return sum(wi * np.exp(-0.5 * ((v - mi) / si) ** 2) / (np.sqrt(2 * np.pi) * si)
                   for wi, mi, si in zip(w, m, s)) / Z

    return cdf, pdf


def sample_velocities(u: np.ndarray, weights, means, sigmas) -> np.ndarray:
    """Inverse CDF of a Gaussian mixture truncated to Omega_v = [-10, 10]."""
    cdf, pdf = _gauss_mixture(weights, means, sigmas)
    return _invert_monotone(cdf, pdf, u, V_MIN, V_MAX)


# --------------------------------------------------------------------------
# families of initial data
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Family:
    """One family of parametric initial data f_v(v; eta) (1 + alpha cos kx)."""
    name: str
    k: float
    # maps one parameter record to (alpha, mixture weights, means, sigmas)
    params: Callable[[dict], tuple]

    @property
    def L(self) -> float:
        return 2.0 * np.pi / self.k


def _landau(eta):
    return eta["alpha"], (1.0,), (0.0,), (eta.get("sigma", 1.0),)


def _two_stream(eta):
    v0, s = eta["v0"], eta.get("sigma", 1.0)
    return eta.get("alpha", 1e-3), (0.5, 0.5), (v0, -v0), (s, s)


def _bump_on_tail(eta):
    return (eta.get("alpha", 0.04), (0.9, 0.1), (0.0, eta["vb"]),
            (1.0, eta.get("sigma_b", 0.5)))


LANDAU = Family("landau", 0.5, _landau)
TWO_STREAM = Family("two_stream", 0.2, _two_stream)
BUMP_ON_TAIL = Family("bump_on_tail", 0.5, _bump_on_tail)
FAMILIES = {f.name: f for f in (LANDAU, TWO_STREAM, BUMP_ON_TAIL)}


def load_particles(family: Family, eta: dict, N: int, quiet: bool = True,
                   seed: int = BASE_SEED, rng: str = "pcg64",
                   sample: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Positions and velocities (each length N, float64) of one sample.

    quiet=True: quiet start on the Hammersley set, x from the base-2 radical
    inverse of l and v from (l + 1/2)/N.  quiet=False: seeded uniform numbers,
    rng="pcg64" (numpy PCG64 stream ``seed``) or rng="philox" (Philox4x32-10
    keyed by ``seed``, counter = (particle, sample); the CUDA loader draws the
    same numbers).
    """
    alpha, w, m, s = family.params(eta)
    if quiet:
        uv, ux = hammersley(N)
    elif rng == "philox":
        ux, uv = philox_uniforms(N, sample, seed)
    else:
        gen = np.random.Generator(np.random.PCG64(seed))
        ux = gen.random(N)
        uv = gen.random(N)
    x = sample_positions(ux, alpha, family.k)
    v = sample_velocities(uv, w, m, s)
    return x, v


def load_batch(family: Family, etas: list[dict], N: int, quiet: bool = True,
               seed: int = BASE_SEED, rng: str = "pcg64") -> tuple[np.ndarray, np.ndarray]:
    """X, V of shape (p, N): sample i uses parameters etas[i] and seed+i
    (rng="pcg64"), or key seed and counter sample i (rng="philox")."""
    X = np.empty((len(etas), N))
    V = np.empty((len(etas), N))
    for i, eta in enumerate(etas):
        if rng == "philox":
            X[i], V[i] = load_particles(family, eta, N, quiet=quiet, seed=seed, rng=rng, sample=i)
        else:
            X[i], V[i] = load_particles(family, eta, N, quiet=quiet, seed=seed + i)
    return X, V


def hammersley_params(p: int, ranges: dict[str, tuple[float, float]],
                      fixed: dict | None = None) -> list[dict]:
    """p parameter records on a Hammersley set over the given box (Sec. 6.1)."""
    names = list(ranges)
    if len(names) == 1:
        cols = [(np.arange(p) + 0.5) / p]
    elif len(names) == 2:
        a, b = hammersley(p)
        cols = [a, b]
    else:
        raise ValueError("at most two varying parameters")
    out = []
    for i in range(p):
        eta = dict(fixed or {})
        for name, col in zip(names, cols):
            lo, hi = ranges[name]
            eta[name] = lo + (hi - lo) * col[i]
        out.append(eta)
    return out


# --------------------------------------------------------------------------
# named workloads (sizes of the benchmark configurations)
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    family: Family
    N: int
    p: int
    Nx: int
    dt: float
    steps: int
    n2: int = 0  # reduced rank 2n (0 = full-order)
    etas: list = field(default_factory=list, hash=False, compare=False)
    quiet: bool = True


def landau_full_order(N=10_000, p=4, Nx=64, dt=0.1, steps=200) -> Workload:
    """Full-order weak Landau damping, alpha in {0.01,0.02,0.03,0.05}, sigma=1."""
    alphas = [0.01, 0.02, 0.03, 0.05]
    etas = [{"alpha": alphas[i % 4], "sigma": 1.0} for i in range(p)]
    return Workload("landau_full_order", LANDAU, N, p, Nx, dt, steps, 0, etas, quiet=False)


def two_stream_reduced(N=100_000, p=64, Nx=128, n2=20, dt=0.05, steps=1000,
                       quiet: bool = False) -> Workload:
    """Reduced two-stream instability, v0 in [2, 3] on a Hammersley set.

    Loading is seeded per sample by default: with a shared quiet start the
    complex snapshot matrix X + iV has sigma_10/sigma_1 ~ 1e-8, so S(Z) is
    numerically singular at 2n = 20 (the full-rank condition on Z fails)."""
    etas = hammersley_params(p, {"v0": (2.0, 3.0)}, {"alpha": 1e-3, "sigma": 1.0})
    return Workload("two_stream_reduced", TWO_STREAM, N, p, Nx, dt, steps, n2, etas, quiet=quiet)


def bump_on_tail_precision(N=1_000_000, p=256, Nx=256, n2=32, dt=0.1, steps=2000,
                           quiet: bool = False) -> Workload:
    """Bump-on-tail, beam mean vb in [4, 5], 10 % beam of width 0.5 (seeded loading)."""
    etas = hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})
    return Workload("bump_on_tail_precision", BUMP_ON_TAIL, N, p, Nx, dt, steps, n2, etas,
                    quiet=quiet)


def particles(w: Workload, seed: int = BASE_SEED) -> tuple[np.ndarray, np.ndarray]:
    return load_batch(w.family, w.etas, w.N, quiet=w.quiet, seed=seed)


# --------------------------------------------------------------------------
# random test matrices
# --------------------------------------------------------------------------
def random_orthonormal_complex(N: int, n: int, seed: int = BASE_SEED) -> np.ndarray:
    """Column-orthonormal complex N x n matrix (QR of a Gaussian matrix)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n))
    Q, _ = np.linalg.qr(A)
    return Q


def random_complex(shape, seed: int = BASE_SEED, scale: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def random_positions(p: int, N: int, L: float, seed: int = BASE_SEED,
                     spread: float = 1.0) -> np.ndarray:
    """Uniform positions on [-(spread-1)/2 L, (spread+1)/2 L): unwrapped when spread > 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.random((p, N)) * spread - 0.5 * (spread - 1.0)) * L


def random_velocities(p: int, N: int, seed: int = BASE_SEED) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.standard_normal((p, N))
