"""GB300-native SpMV engine (y = alpha*A*x + beta*y over CSR/ELL/COO/HYB/BSR/SELL).

The compute path lives in the CUDA shared library built from ``csrc/``;
this package only marshals arguments to its C ABI (see ``binding``).
"""
