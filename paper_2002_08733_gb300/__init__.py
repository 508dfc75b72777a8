"""GB300-native matrix-free DG time-domain Maxwell solver (arXiv 2002.08733).

The compute path is the CUDA library libdgmax.so (C ABI in include/dgmax.h);
``paper_2002_08733_gb300.dgmax`` is its thin Python binding and
``paper_2002_08733_gb300.build`` compiles it for sm_103a.
"""
