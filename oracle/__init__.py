"""CPU oracle for the single-pass mesh + 3DGS rasterizer and the proxy-mesh
binding/deformation of UniMGS (arXiv 2601.19233).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the benchmark's CPU-baseline leg may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or executes
anything here, and this package imports nothing from the product path.

Layout:
  canonical.py  the definitional decisions in canonical IEEE float32 (each op
                rounded separately, no FMA): projected Gaussian pixel rects,
                triangle snapping / integer edge functions / sample coverage,
                depth keys, tile lists and their sort order.
  sh.py         real spherical harmonics from their general definition (fp64).
  render.py     the per-pixel composite of Sec. 3.2 (Eq. 1-2, 7-11) in fp64,
                with the soft-edge sample coverage as an option.
  deform.py     per-face frames, per-vertex polar transforms and the Gaussian
                update of Eq. 12-13 in fp64.
  bind.py       brute-force Gaussian-centric ray-cast binding (Sec. 3.3) and
                the closest-point fallback, canonical float32.
  grad.py       fp64 autograd gradient of the composite (through soft-edge
                coverage too) and a finite-difference helper.
  layers.py     the separate-pass baseline of Sec. 4.1 / Fig. 5b (two layers
                composited per pixel by their expected depths), fp64.
"""
