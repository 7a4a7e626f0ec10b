"""ORACLE -- test infrastructure only.

Plain FP64 CPU references for the branched dual-regularized LQR problem of
"Rake-Compress Riccati Recursions for Parallel Scenario-Tree Model Predictive
Control".  Only the test-suite, the smoke check and the benchmark's CPU-baseline
leg may import anything from this package.  Nothing here is shared with, or
imported by, the CUDA solver.

Contents
  riccati.py  -- ctypes wrapper of tlqr_oracle.c: the sequential tree Riccati
                 recursion and the KKT residual / backward error.
  dense.py    -- the KKT system eq. (kkt) assembled densely and solved directly
                 (brute force for small trees), plus the node-control problem of
                 eq. (node-lagrangian) assembled the same way.
  ops.py      -- per-operation references: condensation eq. (edge-components),
                 rake fold eq. (terminal-fold), compress composition
                 eq. (compress-intermediates)-(composition), reconstruction
                 eq. (value-reconstruction), local factor eq. (FW), (factor-local).
  plan.py     -- the structural rake/compress schedule of Sec. X-A taken
                 literally, with the dependency levels of eq. (earliest-level)
                 and the readiness-weighted reduction of eq. (readiness-code-data).
"""
