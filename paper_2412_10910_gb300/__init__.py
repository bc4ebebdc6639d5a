"""GB300 non-nested matrix-free multigrid (arXiv 2412.10910) behind a small C interface.

`paper_2412_10910_gb300.nnmg` is the Python binding of libnnmg.so (include/nnmg.h);
importing it loads the CUDA library and raises if it has not been built.
`paper_2412_10910_gb300.build` compiles the library for sm_103a.
"""
__all__ = ["nnmg", "build"]
