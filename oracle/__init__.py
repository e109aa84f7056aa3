"""FP64 CPU oracle of the HDG trace-solver hot path -- TEST INFRASTRUCTURE.

A plain, slow, obviously-correct restatement of what the hot path computes,
written from Welter & Nguyen, "Preconditioning Techniques for Hybridizable
Discontinuous Galerkin Discretizations on GPU Architectures" (arXiv
2512.13619).  Every function cites the section / equation it follows.

Only the test-suite, `__graft_entry__.smoke()` and the `cpu_baseline` leg /
`--impl reference` arm of `bench.py` may import this package.  The CUDA
library shares no code with it; both consume the seeded inputs of the
separate `hdg_inputs` package.

Pins (see tests/test_oracle_*.py): manufactured-solution convergence rates,
polynomial patch test, equality with the monolithic dense solve, symmetry of
the Poisson/elasticity trace matrix, ASM blocks = R_e K R_e^T, polynomial
exactness on matrices with few distinct eigenvalues, harmonic Ritz values
against numpy eigenvalues, GMRES against a sparse direct solve.
"""
