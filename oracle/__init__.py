"""FP64 CPU oracle of the variational (Galerkin) FFT solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow restatement of the
method of Lucarini & Segurado, "On the accuracy of spectral solvers for
micromechanics based fatigue modeling" (arXiv:1806.10599), written from the
paper in numpy FP64.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import it; the CUDA library never does, and shares
no code, table or constant with it.

Modules
  spectral   frequencies, the projections G^ and G^' (Sect. 2.2), the
             equilibrium operator and its tangent form (Eqs. eql_discrete3,
             newlinop)
  materials  rotations, cubic/isotropic stiffness, St.Venant-Kirchhoff and
             the FCC crystal-plasticity return map with its consistent tangent
             (Sect. 3.2, Eq. gamma_dot)
  solver     Newton-Raphson with conjugate-gradient linear solves (Sect. 2.1,
             Eqs. F_dif, P_dif, linequil2), mixed macroscopic control
  fips       fatigue indicator parameters (Sect. 3.3, Eqs. eqplas,
             strainenergy, Pmax) and the per-grain Fatemi-Socie parameter

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, brute force or finite differences, except the
crystal-plasticity polycrystal fields and the FIPs, which are "parity
unpinned" beyond the single-voxel checks of the return map and the
single-crystal reduction of a whole polycrystal run (no value printed in the
paper can be reproduced without the FEM reference).
"""
