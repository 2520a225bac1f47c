"""pi/12 piecewise trigonometry (arXiv 2502.10831) on GB300: thin Python layer
over the C-ABI CUDA library ``libptrig``."""
