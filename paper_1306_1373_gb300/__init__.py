"""GB300 (sm_103a) Cordic-based Loeffler DCT image codec.

The compute path lives in ``libdctgb.so`` (C ABI, ``include/dctgb.h``),
built from ``csrc/`` by ``build.build()``; ``dctgb`` is its thin ctypes
binding.
"""
