"""GB300-native free-hand ultrasound volume reconstruction (arXiv 2412.00058).

The compute path -- pose-tracked pixel-nearest-neighbour (or trilinear)
insertion of B-mode frames into a voxel volume, normalisation + 3x3x3 hole
filling, and the depth-band (VPI) projection -- is hand-written CUDA for
sm_103a behind the C ABI declared in ``include/usvol.h``.  ``usvol`` is the
thin ctypes binding to that library; ``synth`` makes seeded synthetic
inputs.  Importing this package loads nothing; the first call into
``usvol`` loads ``libusvol.so`` and raises if it is missing.
"""
__all__ = ["usvol", "synth"]
