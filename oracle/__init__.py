"""FP64 CPU oracle for the collision-resolving Stokes-sphere mobility path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or constants with the CUDA library; the two meet only through
the seeded input generators, which hold none of the method's arithmetic.

Every routine here is a plain, slow restatement of a passage of Yan, Corona,
Malhotra, Veerapaneni & Shelley, "A scalable computational platform for
particulate Stokes suspensions" (arXiv 1909.06623), cited by section and
equation label.  Where the paper is silent, garbled or inconsistent the module
docstring of the routine states the reading taken.

Modules
  sph       -- Gauss-Legendre x uniform grid (Sec. 5.4), Y_n^m and P_n^m
               (Sec. 4.2), VSH basis V, W, X (Sec. 4.2), analysis / synthesis.
  layer     -- kernels G and T and operators S, K (Sec. 4.1), the exterior
               single-layer VSH field of eq. ssgext and its traction (Sec. 4.2),
               self / near / far parts of the layer operators (Sec. 4.2, 5.1).
  mobility  -- rho, L, GMRES on eq. rigidbodyrho, velocity extraction (Sec. 4.1).
  lcp       -- contacts and D (Sec. 3.1-3.2), BBPGD (Algorithm 1), brute-force
               LCP enumeration, one collision-resolved Euler step (Sec. 3.2).
"""
