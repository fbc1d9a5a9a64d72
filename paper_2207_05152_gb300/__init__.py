"""DLIC on GB300: deep lossless image coding with a causal density network,
a fixed-point frequency table and interleaved rANS, encoded all pixels at once
and decoded as a wavefront, all in CUDA kernels for sm_103a behind the C ABI
of include/dlic.h.

Importing the package does not load the CUDA library; the first coding call
does, and fails loudly when libdlic.so has not been built."""

__all__ = ["model", "codec", "build"]
