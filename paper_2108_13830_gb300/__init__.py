"""GB300 (sm_103a) hot path of CNN variational Monte Carlo for the J1-J2 model.

The computation lives in libvmc.so (C ABI: include/vmc.h); `binding`
marshals torch tensors into it and `inputs` generates seeded synthetic
workloads.  Importing the package loads nothing; `binding.lib()` loads the
library on first use and raises if it has not been built.
"""
__all__ = ["binding", "inputs", "build"]
