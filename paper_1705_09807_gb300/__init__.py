"""GB300-native (sm_103a) fused time step of the filtered LES lattice Boltzmann MHD model of
Flint & Vahala (arXiv:1705.09807).

``paper_1705_09807_gb300.lbmhd`` is the Python binding of the C-ABI library
``liblbmhd.so`` (built from ``csrc/``); it loads the library on first use and raises if it
is missing.  ``paper_1705_09807_gb300.inputs`` builds seeded synthetic initial conditions.
"""
