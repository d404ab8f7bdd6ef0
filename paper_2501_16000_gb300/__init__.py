"""GB300-native Onsager-Regularized lattice Boltzmann (D2Q9) stream-collide.

The compute path is the CUDA library ``liboreg.so`` built from ``csrc/``;
``binding`` is its thin ctypes binding (same names as the C ABI in
``include/oreg.h``), ``engine`` holds the ``Lattice`` wrapper, ``batch`` the
batched path and ``serve`` the continuous-batching request loop.
``workloads`` holds only seeded input generators.

Importing the package loads nothing; the library is opened on first use and a
missing or unbuilt library raises instead of falling back to anything else.
"""

__all__ = ["binding", "engine", "batch", "serve", "workloads", "build"]
