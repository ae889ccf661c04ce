"""B300-native (sm_103a) QAOA statevector hot path for QUBO problems.

Submodules:
  qaoa       - ctypes binding of the C ABI (include/qaoa.h); loads libqaoa.so
  autograd   - torch.autograd.Function around qaoa_grad
  instances  - seeded synthetic QUBO instances (inputs only)
  build_lib  - nvcc build of libqaoa.so

The package import itself is light; `qaoa` loads the CUDA library on first
import and fails loudly if it is missing.
"""
