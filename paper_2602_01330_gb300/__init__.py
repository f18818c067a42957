"""GB300-native quantum-classical dual-kernel Gram engine (MPS build, transfer-chain
Gram with fused RBF kernel and linear mix) behind the C ABI declared in include/dualk.h.

``synthetic`` draws seeded inputs; ``dualk`` is the ctypes binding of libdualk.so.
"""
