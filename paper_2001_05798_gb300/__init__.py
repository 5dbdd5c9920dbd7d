"""GB300-native AMG-preconditioned CG solver for steady groundwater flow.

The solver (assembly, smoothed-aggregation setup, V-cycle, PCG) is CUDA code
for sm_103a behind the C ABI declared in ``include/gw.h``; ``gw`` is the thin
ctypes binding over it and ``workload`` draws the seeded synthetic inputs.
"""
__all__ = ["gw", "workload"]
