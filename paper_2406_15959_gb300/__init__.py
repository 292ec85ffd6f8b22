"""GB300-native nonoverlapping domain decomposition for extreme learning machines.

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through :mod:`paper_2406_15959_gb300.elm_ddm`.  :mod:`paper_2406_15959_gb300.workload`
generates seeded synthetic inputs and has no dependency on the library.
"""
__all__ = ["workload", "elm_ddm"]
