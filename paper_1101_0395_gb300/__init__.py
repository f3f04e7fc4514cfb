"""GB300-native exact k-means colour quantization (Weighted Sort-Means).

``kq`` is the binding of the C ABI in include/kq.h (libkq.so, CUDA sm_103a);
``synth`` makes the seeded synthetic input images.
"""
