"""GB300-native Lennard-Jones force over a sorted Verlet pair list.

The compute path lives in a C-ABI CUDA library (``csrc/``, header
``include/lj_gb300.h``); ``lj`` is its thin Python binding.  Importing this
package loads nothing: ``inputs`` (seeded workloads) is usable without a GPU,
and the binding loads the shared library on first use.
"""
