"""GB300-native hot path of the Fokker-Planck central-moment LBM for thermal convection.

The fused collide-and-stream step of the coupled flow (D2Q9 / D3Q27) and energy (D2Q9 / D3Q15)
lattices of Schupbach & Premnath (arXiv 2504.09041), as hand-written sm_103a CUDA behind the C ABI
of include/lbm.h (liblbm.so) and the thin binding in ``lbm``.
"""
