"""Plain FP64 CPU oracle of the one-step ADER-WENO constrained-transport MHD scheme
(Balsara, Florinski, Garain, Subramanian & Gurski, arXiv 1905.02504).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call or execute this package.  Only the tests, the
``__graft_entry__.smoke()`` check and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code, tables or helpers with the CUDA
path; both sides only share the seeded input generators in
``paper_1905_02504_gb300.inputs``, which hold none of the method's arithmetic.

Every routine follows the paper's definitions step by step, per zone, in FP64,
vectorised over zones with numpy only where the per-zone arithmetic is unchanged:

  refelem   -- serendipity / temporal Lagrange bases, R matrix (Sec. V.b-c, App. B-D)
  quadrature-- Gauss-Legendre rules and the printed face rules (App. A)
  mesh      -- cubed-sphere geodesic mesh, log radial shells, isoparametric map,
               zone moments (Sec. II, Eqs. 3.2-3.3, 5.2-5.5)
  weno      -- WENO-AO reconstruction in the Taylor basis (Sec. III, Eqs. 3.1-3.4)
  divfree   -- divergence-free reconstruction of B by KKT (Sec. IV, Eqs. 4.1-4.15)
  ader      -- ADER-CG predictor in mapped coordinates (Sec. V, Eqs. 5.20-5.29, C.34-C.36)
  corrector -- HLL face fluxes, multidimensional edge EMFs, FV + Yee CT update
               (Sec. II.c Eqs. 2.5-2.6, Sec. VI)
  step      -- the full step, CFL time step and div B diagnostic

Parity status of each part is listed in its module header ("pinned by" /
"parity unpinned").
"""
