"""GB300-native conjugate-gradient solver for sparse SPD systems in CSR form.

The hot path (one SpMV, two dot products and three axpy updates per CG
iteration, the case study of the paper's Section IV) runs in hand-written
sm_103a CUDA kernels behind the C-ABI library ``libgbcg.so``; ``gbcg`` is its
ctypes binding.  ``problems`` generates the seeded synthetic inputs.

Importing the package loads nothing native; ``gbcg`` loads the library on
first use and raises if it has not been built.
"""
__all__ = ["gbcg", "problems"]
