"""GB300-native hot path of the Parallel Gaussian Source Finder.

A bank of separable 3D Gaussian filters over an HI cube, window mean and
standard deviation of each filtered cube, the threshold mean + k*std and the
OR of all filters into a packed mask (Westerlund & Harris, Eq. 2 and
Sec. 3.3), as CUDA kernels for sm_103a behind the C ABI of include/sf.h.
"""
from .sf import (BatchSourceFinder, SectionedSourceFinder, Server, SfError, SourceFinder,  # noqa: F401
                 fp32_peak, lib, words_to_bits)
