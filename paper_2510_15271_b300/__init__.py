"""B300-native Levenberg-Marquardt bundle adjustment (cuSfM's BA iteration).

The solver lives in the CUDA library ``libba.so`` behind the C ABI declared
in ``include/ba.h``; ``paper_2510_15271_b300.ba`` is the thin ctypes binding.
``paper_2510_15271_b300.scenes`` synthesises seeded input problems.
"""
