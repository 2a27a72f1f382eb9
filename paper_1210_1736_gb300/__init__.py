"""GB300-native nested-grid particle-mesh gravity step (Superbox-10).

The compute path is libpm.so (hand-written CUDA for sm_103a behind the C ABI
in include/pm.h); `pm` is its ctypes binding, `workloads`/`synth` hold the
seeded synthetic inputs.
"""
from . import pm  # noqa: F401
