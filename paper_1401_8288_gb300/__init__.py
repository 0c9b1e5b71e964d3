"""GB300-native X-stage (cross-multiply and integrate) for FX radio correlators.

The compute path is the C-ABI library built from ``csrc/`` (hand-written
sm_103a CUDA kernels); ``xcorr`` is its thin Python binding.  ``synth`` holds
the seeded synthetic input generators and ``costmodel`` the paper's sizing
equations.  Importing this package loads nothing; the binding loads the
library on first use and fails loudly when it is missing.
"""

__all__ = ["synth", "costmodel", "xcorr"]
