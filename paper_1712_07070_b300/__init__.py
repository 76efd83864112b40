"""B300-native GAMER-2 patch-group hydro update (MUSCL-Hancock + PLM + HLLC on
an AMR hierarchy of 8^3 patches), hand-written CUDA for sm_103a behind a C ABI.

Importing the package loads nothing; ``paper_1712_07070_b300.amr_hydro``
loads the compiled library and fails loudly if it is missing.
"""
