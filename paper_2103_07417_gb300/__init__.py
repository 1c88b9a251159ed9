"""GB300-native adaptive ray tracing of Kerr black-hole images (Gelles et al. 2021).

The compute path is the CUDA library ``lib/libart_gb300.so`` (sources in ``csrc/``, C-ABI in
``include/art.h``); ``art`` is its thin ctypes binding.
"""
