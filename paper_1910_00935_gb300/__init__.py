"""GB300-native differentiable MLS-MPM (DiffTaichi's diffmpm hot path, Section 4.1).

Submodules:
  scenes -- seeded synthetic inputs (no simulation arithmetic)
  mpm    -- ctypes binding of the C-ABI library libmpm.so and the torch autograd wrapper
  build  -- compiles libmpm.so for sm_103a
Importing the package does not load the CUDA library; ``mpm`` does, and fails loudly
when it is missing.
"""
__all__ = ["scenes"]
