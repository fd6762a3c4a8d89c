"""GB300-native short-range TreePM path (Ishiyama, Nitadori & Makino, SC12).

The compute path is the CUDA library libtreepm_sr.so (C-ABI in
include/treepm_sr.h); this package only marshals arguments to it.
"""
__all__ = ["inputs"]
