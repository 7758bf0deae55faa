"""GB300 (sm_103a) implementation of the hot path of the multilevel
local-expansion Metropolis-Hastings electrostatics method of Saunders, Grant &
Mueller (arXiv 2006.16622).

The compute path is the CUDA library ``libmcfmm.so`` behind the C ABI of
``include/mcfmm.h``; :mod:`.mcfmm` is its thin binding and :mod:`.workloads`
draws seeded synthetic inputs.  Importing the package does not load the
library; :func:`mcfmm.load` does, and raises when it is missing.
"""
