"""GB300-native exact fixed-radius neighbour search by sorting (SNN).

The compute path lives in the CUDA library ``libsnn.so`` (sources under
``csrc/``, C ABI in ``include/snn.h``); ``snn`` is its thin ctypes binding.
Importing this package loads nothing; ``paper_2212_07679_gb300.snn`` loads the
library and fails loudly when it is missing.
"""
__all__ = ["snn", "workloads", "build"]
