"""GB300-native batched level-wise B+ tree point search.

The compute path is a C-ABI CUDA library (``csrc/``, built for sm_103a);
``btree`` is its thin ctypes binding.  Importing the package itself loads
nothing native; importing ``paper_2604_21117_gb300.btree`` loads the library
and raises if it has not been built.
"""
