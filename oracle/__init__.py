"""Plain FP64 CPU oracle for the infinite-cell Clenshaw-Curtis SQ density / energy / stress.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package. It shares no code with the
CUDA library (paper_2006_03697_gb300) and never imports it; both take their inputs
from the seeded generators in workloads/.

Modules
  sq_oracle     the SQ sweep of Sec. 4 (nodal Hamiltonians, Chebyshev recurrence,
                moments, Clenshaw-Curtis coefficients, Fermi bisection, contraction)
  dense_k       k-integrated dense diagonalisation of the periodic grid Hamiltonian
                (infinite-crystal limit, density-matrix stress of Eq. (ON:Stress),
                Mermin free energy under homogeneous strain, Eq. (stressdefinition))
  free_electron closed forms for V_eff = 0 and no projectors (Brillouin-zone integrals
                and the exactly separable truncated region)
  green_kubo    Green-Kubo shear viscosity of a stress time series (Eq. viscosity)
  per_node      the per-node spectral bounds mode (chi_q, zeta_q of each H_q)
  gauss_sq      Gauss Spectral Quadrature of the density (Lanczos from e_q per node)
"""
