"""GB300 two-population phase-field lattice Boltzmann library (arXiv 1812.00118).

The compute path is the C-ABI shared library ``liblbm`` (CUDA, sm_103a) built
from ``csrc/``; ``lbm`` is its thin ctypes binding.  Import submodules
explicitly (``from paper_1812_00118_gb300 import lbm``); this package
initialiser loads nothing so that ``inputs`` can be used without a GPU.
"""
