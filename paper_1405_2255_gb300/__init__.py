"""GB300-native fast multipole method for unsoftened N-body gravity
(Dehnen, "A fast multipole method for stellar dynamics", arXiv 1405.2255).

The compute path is the CUDA library built from ``csrc/`` (``build.py``); the
module ``gb3fmm`` is its Python binding and ``inputs`` draws seeded synthetic
particle sets.  Importing the package loads nothing on the GPU.
"""
__all__ = ["gb3fmm", "inputs", "build"]
