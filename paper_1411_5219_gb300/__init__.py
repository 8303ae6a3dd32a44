"""GB300-native even-odd Wilson / twisted-mass Wilson Dslash and CG solver.

The compute path is the CUDA library ``libqcd.so`` (sm_103a) behind a C ABI
declared in ``include/qcd.h``; ``paper_1411_5219_gb300.qcd`` is its thin
ctypes binding.  ``synthetic`` draws the seeded inputs.
"""
