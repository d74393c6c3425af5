"""GB300 (sm_103a) implementation of the one-step ADER-WENO constrained-transport MHD
scheme on a radially extruded cubed-sphere mesh of isoparametric hexahedra
(Balsara, Florinski, Garain, Subramanian & Gurski, arXiv 1905.02504).

The compute path is the CUDA library ``lib/libgeomhd.so`` (C ABI in
``include/geomhd.h``); ``geomhd`` is its thin ctypes binding and ``inputs`` holds
the seeded synthetic initial data.
"""
