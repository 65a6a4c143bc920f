"""GB300-native single-pass mesh + 3D Gaussian Splatting rasterizer and
proxy-mesh binding/deformation (UniMGS, arXiv 2601.19233).

The compute path is the C-ABI library ``libumgs.so`` (hand-written sm_103a
CUDA kernels, see ``csrc/``); ``umgs`` is its thin Python binding.
"""
