"""GB300-native Piacsek-Williams advection (su, sv, sw source terms).

The compute path is a CUDA library for sm_103a behind a C ABI
(``include/pw.h``); ``paper_2107_13500_gb300.pw`` is its thin Python
binding. Importing the package itself loads nothing: ``synth`` (input
generation) is usable without a GPU or a built library.
"""
