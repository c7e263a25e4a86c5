"""GB300-native NLPR multiband fusion: CUDA library (libfuse.so, C-ABI in include/fuse.h)
plus a thin ctypes binding (fuse.py), an in-tree build (build.py) and seeded synthetic
problems (synth.py)."""
