"""GB300-native (sm_103a) multiple-resolution scalar path of arXiv:1805.03426.

Divergence-free refinement of a coarse staggered velocity onto a dense grid and
the second-order finite-volume advection-diffusion step of a scalar, as CUDA
kernels behind the C-ABI in include/mr.h; ``mr`` is its ctypes binding and
``synth`` draws the seeded synthetic inputs.
"""
