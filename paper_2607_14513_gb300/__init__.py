"""GB300-native block-texture coding of 3DGS spherical-harmonic colour.

The codec itself lives in libgsc.so (CUDA for sm_103a, C ABI in include/gsc.h);
``gsc`` is its thin Python binding and ``synthetic`` draws seeded input scenes.
"""
