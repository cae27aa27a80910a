"""QFactor-Sample instantiation on GB300 (sm_103a).

The compute path is the C-ABI library ``libqfs.so`` built from ``csrc/``;
``qfs`` is its Python binding.  ``workloads`` holds the seeded input
generator.  Importing the package loads nothing; the binding loads the
library on first use and raises if it is missing.
"""
