"""The conditioning behind the precision reading of the 200-step gate: the
FP64 oracle, started from coefficients Z rounded to FP32 (a relative change
of at most 2^-24 per entry), leaves its own unperturbed run by more than the
1e-6 gate in the Hamiltonian within 200 steps of a randomly loaded
bump-on-tail case, while one step stays far inside it.  The PIC force is
piecewise constant in the positions (Sec. 2.1), so a particle that changes
cell changes it by a finite amount; no form whose state carries FP32
rounding can follow the FP64 trajectory to 1e-6 over such a horizon."""
import numpy as np

import workloads as W
from oracle import csvd, pic, reduced

GATE = 1e-6


def test_fp32_rounding_of_the_start_moves_the_oracle_past_the_gate():
    N, p, n, Nx, dt, steps = 2000, 8, 4, 64, 0.1, 200
    etas = W.hammersley_params(p, {"vb": (4.0, 5.0)}, {"alpha": 0.04, "sigma_b": 0.5})
    X0, V0 = W.load_batch(W.BUMP_ON_TAIL, etas, N, quiet=False)
    U, Z, _ = csvd.csvd_init(X0, V0, n)
    Z32 = Z.astype(np.float32).astype(np.float64)
    assert np.max(np.abs(Z32 - Z) / np.abs(Z).max()) <= 2.0 ** -24
    g = pic.make_grid(N, Nx, W.BUMP_ON_TAIL.L)
    _, _, tro, _ = reduced.run(U, Z, dt, steps, g, warm_start=True)
    _, _, trp, _ = reduced.run(U, Z32, dt, steps, g, warm_start=True)
    dev = np.abs(trp[:, :, 1] - tro[:, :, 1]) / np.abs(tro[:, :, 1])
    assert dev[0].max() < 0.1 * GATE
    assert dev.max() > 10 * GATE
