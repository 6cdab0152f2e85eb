"""FP64 CPU oracle of the parametric particle Vlasov-Poisson reduced model.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of what arXiv 2201.05555 (Hesthaven, Pagliantini, Ripamonti)
defines, written with numpy in float64.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The CUDA library never calls it and it
never calls the CUDA library; the two share no code.  The only shared module
is ``workloads`` (seeded input generation, no method arithmetic).

Modules
-------
pic        geometric PIC: P1 hats, deposit, periodic Poisson, gather, energies (Sec. 2.1)
full_order Stormer-Verlet full-order step (Sec. 5, eq. sv_full_order)
reduced    dynamical ortho-symplectic reduced model in the paper's real 2N x 2n
           form: gradients, basis velocity, Cayley retraction, tangent
           velocity, partitioned RK2 step (Sec. 3.2, Sec. 5)
csvd       truncated complex SVD initialisation (Sec. 3.2, Algorithm 2)
deim       DEIM-indexed gradient of the DMD-DEIM Hamiltonian (Sec. 4.2, eq. grHDD)
diagnostics damping/growth-rate fits, Hamiltonian error, manifold residuals (Sec. 6)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, invariants, special cases
or brute force, except ``diagnostics.fit_rate`` on the paper's own figures
(figures are not available; pinned only through the Landau rate of the full
model).
"""
from . import pic, full_order, reduced, csvd, deim, diagnostics  # noqa: F401
