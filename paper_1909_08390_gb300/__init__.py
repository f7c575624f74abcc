"""GB300-native IMEX finite-difference lattice Boltzmann hot path.

``paper_1909_08390_gb300.fdlb`` is the binding of the C-ABI library
``libfdlb.so`` (sm_103a CUDA kernels).  ``workloads`` holds the seeded
synthetic problem definitions.  Importing the package loads nothing; the
library is loaded on first use of ``fdlb``.
"""
