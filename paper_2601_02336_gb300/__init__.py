"""GPU (sm_103a) hot path of an SMC sampler with a NUTS transition kernel for
gravitational-wave inference (arXiv:2601.02336).

`inputs` holds the seeded synthetic workloads; `api` the Context class over
the C ABI of libsharpy (include/sharpy.h). Submodules are imported on demand
(`from paper_2601_02336_gb300 import api`), so importing the input recipes
does not load the CUDA library.
"""
