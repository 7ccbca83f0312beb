"""FP64 CPU oracle for tree-level NLO matrix elements and FKS subtraction.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package: only the
tests, the smoke check and the CPU-baseline leg of the benchmark do.  It shares
no code with the CUDA path (no kernels, headers, tables or generators); the only
common dependency is the seeded input module ``synth``.

What it computes (hep-ph background of arXiv:2503.07439):
  * tree-level squared matrix elements as the plain definition -- every Feynman
    diagram evaluated with explicit 4x4 Dirac matrices, explicit helicity
    spinors and polarisation vectors, and an explicit SU(3) colour tensor per
    diagram; |M|^2 = sum over helicities and over all colour assignments
    (Sec. 2.1, Eq. (born); Sec. 2.2, Eq. (real); Sec. 4.2: Born, real and
    counterterms are all tree-level amplitudes);
  * colour-correlated and spin-correlated Born matrix elements;
  * the FKS real-minus-counterterm weight in the sector parametrisation
    (Sec. 2.2 subtraction schemes; Sec. 4.2 FKS sectors; Algorithm 2 evaluates
    Born, real, soft and collinear terms unconditionally, then masks them);
  * for e+e- -> u ubar the analytic virtual plus integrated FKS counterterms;
  * infrared-safe cuts applied to each term at its own kinematics (Algorithm 2's
    passCuts(a, p)): heavy-quark p_T and rapidity, e+e- thrust and thrust axis.

The paper prints no formulas for any of this; every formula here is standard
physics restated in the modules' docstrings, and each is pinned by the tests in
``tests/test_oracle_*.py`` (closed forms, traces, gauge invariance, symmetry,
colour conservation, soft/collinear ratios, phase-space volumes, K-factor).
"""
