"""B300-native DGSEM residual and SSP-RK3 stage (arXiv 2605.26388, Sec. 3.1 and App. A-B).

The compute path is the C-ABI library ``libdgsem.so`` (hand-written sm_103a CUDA); the
Python layer only marshals arguments.  Import ``paper_2605_26388_b300.dgsem`` for the
binding; importing this package itself loads nothing.
"""
__all__ = ["dgsem", "workloads"]
