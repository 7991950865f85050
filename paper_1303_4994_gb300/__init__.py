"""GB300-native APAX codec: block encode/decode of integer and float arrays and
the profiler sweep of Wegener, arXiv 1303.4994 (Sec. 4 profiler, Sec. 6
encoder and bit packer), as sm_103a CUDA kernels behind the C ABI of
include/apax.h.  ``apax`` is the Python binding; ``synth`` draws the seeded
synthetic inputs; ``build`` compiles the library in-tree."""
from . import apax, synth  # noqa: F401
