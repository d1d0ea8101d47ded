"""GB300-native Euler characteristic curves of gray-scale images (Heiss & Wagner).

The compute path is the CUDA library ``libecc_gb300.so`` behind the C ABI in
``include/ecc.h``; ``paper_1705_02045_gb300.ecc`` is its Python binding.
"""
