"""Plain FP64 CPU oracle for the EOFA / optimal domain-wall hot path.

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU-baseline leg
of the benchmark may import this package. The library's CUDA path never calls it, and
this package imports nothing from the CUDA binding; the two share only the seeded input
generators of ``paper_1710_09621_gb300.inputs``.

Everything here is written for obvious correctness, not speed: whole-lattice numpy
arrays in complex128, np.roll for the nearest-neighbour shifts, explicit 4x4 gamma
matrices, dense Ns x Ns fifth-dimension matrices and numpy.linalg for inverses and
determinants. Each function cites the passage of Chen & Chiu, "Mass Preconditioning
for the Exact One-Flavor Action in Lattice QCD with Domain-Wall Fermion"
(arXiv:1710.09621) that it follows, as Section / Eq.(label).

Pins (see tests/test_oracle_*.py): gamma5-hermiticity, gauge covariance, the free-field
momentum-space closed form, the EOFA determinant identities of Eq.(det_minus),
Eq.(det_plus), Eq.(m1m2_m1m4), Eq.(m1m2_m3m2), Eq.(new_MP) and Eq.(old_MP) by brute force
on a 2^4 x Ns=4 lattice, rank-one mass dependence Eq.(delta_ij)/(k_ij), the true residual of
the solver, finite differences of the action for the force, and phi^dag X phi = eta^dag eta
for the heat-bath.
"""
