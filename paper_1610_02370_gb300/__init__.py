"""GB300-native hot path of twisted-mass DD-alpha-AMG (arXiv:1610.02370).

The compute path is the C-ABI library ``libddtm.so`` (hand-written sm_103a CUDA
kernels, header ``include/ddtm.h``).  ``paper_1610_02370_gb300.ddtm`` is the thin
ctypes binding with the same entry-point names; importing it loads the library
and raises if it has not been built.  ``synth`` draws the seeded synthetic
inputs.
"""
