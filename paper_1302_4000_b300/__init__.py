"""B300-native all-versus-all cRMSD (ClusCo, arXiv 1302.4000).

The CUDA path lives in ``libclusco.so`` (C-ABI, declared in ``include/clusco.h``);
``paper_1302_4000_b300.clusco`` is the thin Python binding over it. Importing
this package is cheap: the shared library is loaded on first use.
"""
__all__ = ["clusco", "ensembles"]
