"""CPU oracle for the HMC hot path of the Hubbard model on the honeycomb lattice.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
complex128 restatement of the method of Krieg, Luu, Ostmeyer, Papaphilippou and
Urbach, "Accelerating Hybrid Monte Carlo simulations of the Hubbard model on the
hexagonal lattice" (arXiv:1804.07195). Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

It shares no code with the CUDA library: the two meet only in the seeded input
generators of the `workloads` module. Every function cites the passage of the
paper it follows. Where the paper is silent or ambiguous the reading taken is
stated beside the code.

Modules:
  lattice     -- honeycomb torus, neighbour and time-shift tables (Section 2)
  fermion     -- M, M^dagger, M M^dagger, dense M, free-field spectrum (Eq. ferm_op)
  free_field  -- M M^dagger + sigma applied and inverted exactly by FFT for a
                 constant field (Eq. ferm_op in plane waves)
  solvers     -- dense LU, CG, single-precision CG, flexible GMRES (Algorithm A.1)
  action      -- log det, pseudofermion action and force, Hasenbusch terms
                 (Eqs. hamiltonian, p_dot, eta_xi, f_chi_i, def_xi_i)
  integrators -- leapfrog, Omelyan, force gradient, nested multi-time-scale
                 Omelyan, Hamiltonian and one MD trajectory (Sections 4 and 5.2)
  ed          -- exact diagonalisation of a small Hubbard cluster (Section 8.1)

Parity status: every function here is pinned by a test under tests/ against a
closed form, a library routine, an invariant or a value the paper prints,
except where its docstring says "parity unpinned".
"""
