"""GB300-native ZipNN codec: byte grouping + chunked Huffman + XOR delta.

The codec runs in hand-written CUDA kernels behind the C ABI of
``libzipnn_gpu.so`` (declared in ``include/zipnn.h``); ``zipnn`` is the thin
ctypes binding.  The native library is loaded lazily on first use.
"""
