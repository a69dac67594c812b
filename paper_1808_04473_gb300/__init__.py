"""GB300-native decentralized feedforward L-MMSE equalization (PD and FD).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through the C ABI declared in ``include/ffeq.h``; ``ffeq`` is the thin
ctypes binding over it.  Importing this package loads nothing: the library is
opened on first use, and every entry point fails loudly if it is missing.
"""
__all__ = ["ffeq", "synth"]
