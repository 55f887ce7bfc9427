"""GB300-native speculative graph colouring (RSOC and two-phase First-Fit).

The compute path lives in the CUDA library ``csrc/`` builds (``libgc.so``);
``gc`` is its thin ctypes binding and ``inputs`` holds the seeded synthetic
graph generators.  Importing the package loads nothing native.
"""
__all__ = ["gc", "inputs"]
