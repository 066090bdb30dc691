"""GB300-native hybrid lattice-Boltzmann / immersed-boundary capillary solver.

The compute path is the CUDA library ``liblbib.so`` (C ABI declared in
``include/lbib.h``); :mod:`paper_2210_06043_gb300.lbib` is its thin ctypes
binding and :mod:`paper_2210_06043_gb300.workloads` the seeded input
generators.  Importing this package loads nothing native.
"""
