"""GB300-native ZNCC + DT + WTA stereo matching (arXiv 2212.00476): the CUDA library
libzncc.so (include/zncc.h) and its thin Python binding.

Importing the package loads nothing; `zncc.lib()` loads the in-tree library and raises if it
has not been built (`python -m paper_2212_00476_gb300.build`). There is no CPU fallback.
"""

__all__ = ["build", "zncc"]
