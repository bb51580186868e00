"""Plain FP64 CPU oracle for the staggered phase-field fracture method.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run anything
in this package.  The product path (the CUDA library and its Python binding) never
imports it and never falls back to it.

What it computes (Luo, "Fast staggered schemes for the phase-field model of brittle
fracture based on the fixed-stress concept", arXiv 2209.07969):

* ``model``      -- pointwise constitutive law: volumetric/deviatoric energy split
                    (Sec. 2, energy split equations), the degraded stress (Eq. for sigma,
                    Sec. 2), AT2 functions (Table 1), the fixed-stress extra stiffness
                    (Sec. 3.3-3.4) and the predicted active energy (Sec. 3.3, with the
                    Delta d > 0 rule of Sec. 3.5).
* ``q1``         -- bilinear (Q1) finite elements on a structured nx-by-ny grid with
                    2x2 Gauss quadrature; assembled sparse (CSR) operators for the weak
                    forms F_u and F_d of Sec. 3.2, plus per-quadrature-point fields.
* ``staggered``  -- semismooth Newton for u, the AT2/history d-solve, the standard
                    staggered scheme (Sec. 3.1, Fig. 1) and the fixed-stress S1/S2/S3
                    schemes (Sec. 3.3-3.5, Table 2), solved with SciPy's sparse direct
                    LU (SuperLU).
* ``monolithic`` -- Newton on the coupled system with the full Jacobian of Sec. 3.2
                    (reference for the converged state of a load step).

Everything is float64 and deliberately unoptimised: vectorised numpy over elements is
the only liberty taken.  The oracle shares no code with the CUDA path.
"""
