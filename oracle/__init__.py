"""Plain FP64 CPU oracle for the space-time multigrid (STMG) hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import or run anything in this
package.  The CUDA library never calls it and shares no code with it; the only
common dependency is the seeded input generator package `synth`.

Every function is a direct, slow, readable restatement of the paper:
  fe1d      -- 1D quadrature rules and Lagrange bases (Section 2, eq. spacetime_discrete)
  timeint   -- dG(k) / cGP(k) time weights and slab systems (eqs. dg-time-weights,
               cg-time-weights, heat-cg-dg, heat-cg-cg, wave-cg-dg, wave-cg-cg)
  space     -- Q_p mass / stiffness on Q1-mapped hexahedra (eq. space-matrices)
  slab      -- slab operator, right-hand side, direct solve, velocity update
  mg        -- transfers (Section 3.2), cell-wise additive Schwarz (eqs. vanka0, vanka),
               V-cycle (Algorithm stmg), relaxation (eq. relaxation), FGMRES
  atonce    -- several heat dG(k) slabs in one system (eq. heat-cg-dg-at-once) and tau-multigrid
               (Algorithm mg-sequence, mgType tau)
  points    -- point values of a finite-element function (goal quantities, Section 4.3)
  conv      -- direct 3D convolution network used for the learned initial guess

Parity status per function is stated in each module header.
"""
