"""FP64 CPU oracle for the MLS field reconstruction (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package.  The library under ``paper_1408_0677_gb300``
never imports it, and it imports nothing from there.

``mls_oracle.c`` is the plain definition (per-pixel weighted least squares in
FP64, Section 3.3 of the paper); this module compiles it with gcc and calls
it through ctypes.  ``space_map.py`` states the space mappings of Section 3.4
(field to RGBA image) in float32 numpy.
"""
from .oracle import VARIANT_MEAN, VARIANT_RIGID, OracleResult, bands, build, mls, mls_variant  # noqa: F401
