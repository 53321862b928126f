"""FP64 CPU oracle for the adaptive multigrid Wilson-Dirac solve.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of the method in Brannick, Brower, Clark, Osborn, Rebbi,
"Adaptive Multigrid Algorithm for Lattice QCD" (arXiv:0707.4018). Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. The product (the CUDA library and its Python
binding) never imports, links or executes anything here, and nothing here
imports the product.

Every floating-point computation is complex128 / float64 with numpy; library
primitives (matmul, LAPACK LU, ARPACK) serve only as single steps. There is no
blocking, fusion or reordering beyond what the paper's definitions state.

Modules
  lattice   -- site, block and coarse-site index maps
  wilson    -- gamma matrices and the Wilson-Dirac operator D (paper, Wilson D
               definition following Eq. 1)
  transfer  -- block Gram-Schmidt, prolongation P and restriction P^dagger
               (Eq. P1 and the adaptive step that appends v_2j, ...)
  coarse    -- Galerkin coarse operator P^dagger D P as a nearest-neighbour
               block stencil (Eq. Galerkin)
  solvers   -- MR smoother, V-cycle (the five steps and Eq. vcycle), coarsest
               exact solve, flexible GCR outer loop
  setup     -- adaptive setup (Eq. relax, Eq. P1, the adaptive passes)
  rng       -- Philox4x32-10 + Box-Muller draws of the setup's random vectors
  spectrum  -- critical mass m_c from the low edge of the spectrum of D

Parity pins: every function is checked by tests that do not re-type it (closed
forms, invariants, special cases, brute force). The adaptive setup beyond its
first pass has no closed form: individual near-null vectors there are
"parity unpinned" and are checked through invariants only (orthonormality,
monotone decrease of ||D v|| / ||v||, MG iteration counts).
"""
