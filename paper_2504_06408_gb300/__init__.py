"""GB300 (sm_103a) semiring SpGEMM: C = A (x).(+) B on CSR over a semiring id.

``spgemm`` holds the Python binding of the C ABI (include/spgemm.h); the
kernels live in ``csrc/`` and are built by ``build.py`` into
``_build/libspgemm.so``.  ``inputs`` draws the seeded synthetic workloads.
The package imports nothing heavy at import time.
"""
