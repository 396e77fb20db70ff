"""Oracle: a plain, slow, FP64 CPU implementation of the space-filling-curve
two-level overlapping Schwarz method (Griebel, Schweitzer, Troska, arXiv 2110.11211).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link
this package: only the tests, the smoke check and the CPU-baseline leg of the
benchmark use it.  It shares no code with the CUDA library; the only module both
sides use is the seeded input generator (`paper_2110_11211_gb300.inputs`), which
holds none of the method's arithmetic.

Modules (each function cites the passage of the paper it follows):
  grid       -- eq. (dof), the finite-difference operator of Sec. 3.3 / Sec. 4
  sfc        -- the d-dimensional Hilbert map of Sec. 3.2 (Skilling's transform)
                and the curve order of Algorithm 1, step 3
  partition  -- eqs. (sloc), (enlarge), (Di), (omegai), (restr) and Lemma 3.1
  schwarz    -- A_i = R_i A R_i^T, A_0 = R_0 A R_0^T (eq. csm), the additive
                preconditioner (eq. addSW, Algorithm 2) and the balanced one (eq. balSW)
  krylov     -- preconditioned CG (Sec. 3.3) and damped Richardson (Algorithm 3)
  exact      -- the plain definition u = A^{-1} f (dense Cholesky / sparse direct)
  adjoint    -- gradients of L = ||u - u_t||^2 through u = A(c)^{-1} f
  combi      -- combination-technique subproblem counts (Sec. 2, Table 1)

Parity status: every function is pinned by the CPU tests in tests/test_oracle_*.py
except the Hilbert curve's orientation convention, which the paper does not fix
(parity unpinned for orientation; bijection and continuity are pinned).
"""
