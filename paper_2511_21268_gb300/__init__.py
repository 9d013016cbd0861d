"""GB300-native matching-based aggregation AMG-PCG for IgA stiffness systems.

The solver lives in a CUDA library behind a C ABI (``include/amg_gb300.h``);
``paper_2511_21268_gb300.amg`` is its thin Python binding and
``paper_2511_21268_gb300.inputs`` builds seeded IgA test systems.
Nothing is loaded at import time.
"""
__all__ = ["amg", "inputs"]
