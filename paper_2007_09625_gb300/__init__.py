"""GB300-native (sm_103a) dual-quantization + Huffman lossy compressor for
FP32 fields, after cuSZ (Tian et al., PACT 2020).

The compute path is the CUDA library ``libgbsz.so`` (C ABI in
``include/gbsz.h``); ``gbsz`` is its Python binding and ``workloads`` the
seeded synthetic input generators.
"""
