"""GB300-native dual-number 3D space-charge PIC (forward-mode AD particle-in-cell).

The compute path is the CUDA library libadpic.so behind the C ABI of
include/ad_pic.h; `adpic` is its ctypes binding and `inputs` holds the seeded
workload recipes. Importing the package loads nothing; the binding loads the
library on first use and raises if it has not been built.
"""
__all__ = ["adpic", "inputs", "build"]
