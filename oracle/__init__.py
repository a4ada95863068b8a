"""FP64 CPU oracle for the discrete Dirichlet-to-Neumann build and solve.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package; the library (paper_1302_5995_gb300) never
does, and shares no code with it.

  o1  -- plain definition: banded Gaussian elimination of the whole five-point
         system, then the one-sided boundary flux (plain C, o1_full.c).
  nd_dense -- the paper's dense nested dissection, step by step (numpy).
  hbs -- the paper's HBS format and its algorithms (numpy).
  closed_form -- exact solutions used to pin the two above.
"""
