"""GB300-native AMR multigrid Poisson solve for electrostatic PIC
(Frey, Adelmann & Locans, arXiv 1812.03689).

The compute path is ``libamrmg.so`` (hand-written sm_103a CUDA behind a C
ABI, declared in ``include/amrmg.h``); ``paper_1812_03689_gb300.amrmg`` is its
thin ctypes binding.  Importing this package itself loads nothing, so the
seeded input generators in ``paper_1812_03689_gb300.inputs`` can be used on
machines without a GPU.
"""
