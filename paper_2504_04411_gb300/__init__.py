"""GB300-native hypothesis-tested progressive kernel estimation (FPPM / VCM+).

The compute path lives in the CUDA library ``libppm.so`` built from
``csrc/``; ``ppm`` is its thin ctypes binding.
"""
