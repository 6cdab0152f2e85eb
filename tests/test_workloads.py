"""Input generators: the counter-based generator against its published
known-answer values, and basic properties of the loaders."""
import numpy as np

import workloads as W


def test_philox4x32_10_known_answers():
    # known-answer vectors of Philox4x32 with 10 rounds (Random123 distribution)
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in cases:
        got = [int(x) for x in W.philox4x32(ctr, key)]
        assert got == want


def test_philox_uniforms():
    ux, uv = W.philox_uniforms(200_000, 3, W.BASE_SEED)
    for u in (ux, uv):
        assert u.min() >= 0.0 and u.max() < 1.0
        assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1 / 12) < 5e-3
    assert abs(np.corrcoef(ux, uv)[0, 1]) < 1e-2
    # sample index and seed select independent streams; the same call repeats
    ux2, _ = W.philox_uniforms(200_000, 4, W.BASE_SEED)
    ux3, _ = W.philox_uniforms(200_000, 3, W.BASE_SEED + 1)
    assert abs(np.corrcoef(ux, ux2)[0, 1]) < 1e-2 and abs(np.corrcoef(ux, ux3)[0, 1]) < 1e-2
    assert np.array_equal(ux, W.philox_uniforms(200_000, 3, W.BASE_SEED)[0])


def test_loaded_moments():
    """Loaded particles follow f0: density (1 + alpha cos kx)/L in x, the
    mixture's mean and variance in v (philox and quiet start)."""
    N = 200_000
    eta = {"v0": 2.5, "sigma": 1.0, "alpha": 0.2}
    fam = W.TWO_STREAM
    for quiet, rng in ((True, "pcg64"), (False, "philox")):
        x, v = W.load_particles(fam, eta, N, quiet=quiet, rng=rng, sample=1)
        assert x.min() >= 0.0 and x.max() < fam.L
        # E[cos kx] = alpha / 2 for the density (1 + alpha cos kx)/L
        assert abs(np.mean(np.cos(fam.k * x)) - 0.1) < 1e-2
        assert abs(v.mean()) < 1e-2
        assert abs(v.var() - (1.0 + 2.5 ** 2)) < 3e-2
