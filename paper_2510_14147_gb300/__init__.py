"""Exact ε-graphs with a cover tree on one GB300 GPU.

The computation lives in the CUDA library built from ``csrc/`` (see
``build.build()``); ``ctgraph`` is its ctypes binding; ``inputs`` draws the
seeded synthetic workloads.  Importing this package loads nothing: the
library is opened on the first call into ``ctgraph``.
"""
__all__ = ["ctgraph", "inputs", "build"]
