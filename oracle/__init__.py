"""Plain FP64 CPU oracle for the componentwise solver-free ADMM.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the CUDA library (it reads the same seeded feeder records and nothing else).

What it computes, with the passage each module follows:

* ``model``      -- the linearized multi-phase OPF (Section II-A: operational
  bounds, power balance, voltage-dependent load model VDLM-1..10, linearized
  power flow with the M^p/M^q matrices, objective sum of pg), written as the
  abstract LP of Eq. (LP_model) and split into fine-grained components
  (bus / line / load / generator) as in Eq. (OurModel).
* ``precompute`` -- row reduction of [A_s | b_s] to full row rank (Section
  IV-B) and the closed-form operators Abar_s, bbar_s of Eq. (closed_2).
* ``admm``       -- Algorithm 1: initialization (Section V-A), the global
  update of Eq. (global_sparse), the local update of Eq. (closed_2), the dual
  update of Eq. (ADMM-3) and the termination test of Eq. (termination);
  plus the LP duality-gap certificate of the iterate.
* ``lp``         -- the centralized LP of Eq. (LP_model) solved by HiGHS
  (scipy), used only to pin the ADMM fixed point on small feeders.

Pins (tests/test_oracle_*.py, CPU only) tie each function to something other
than itself: closed forms, brute-force minimization, a dense KKT solve, SVD
null spaces, an independent phasor derivation of the line and delta-load
equations, hand-solvable feeders and HiGHS.  Items with no such pin:
"parity unpinned" -- the paper's Table V iteration counts (different data).
"""
