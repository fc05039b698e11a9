"""GB300-native HPS direct solver for the 2-D variable-coefficient Helmholtz
impedance problem (arXiv:1812.07167).

The solver is a C-ABI shared library (``include/hps.h``) built from the CUDA
sources in ``csrc/``; ``hps`` is its thin Python binding.  Importing this
package loads nothing; ``from paper_1812_07167_gb300 import hps`` loads the
library and fails loudly if it has not been built.
"""
