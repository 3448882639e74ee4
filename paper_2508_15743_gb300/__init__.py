"""VibeLSD decoding on GB300 (sm_103a): package root.

The CUDA library and its ctypes binding live in `paper_2508_15743_gb300.vibe`; the seeded input
generators in `paper_2508_15743_gb300.dem`. Importing the package itself loads nothing native.
"""
