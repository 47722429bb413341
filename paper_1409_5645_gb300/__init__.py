"""GB300-native free-surface lattice Boltzmann step (D3Q19, FSK/FSL closures).

``paper_1409_5645_gb300.fslbm`` is the binding of the CUDA library's C ABI;
``paper_1409_5645_gb300.cases`` builds seeded synthetic inputs.
"""
