"""GB300-native electromagnetic shower transport (AdePT, arXiv 2209.15445).

The compute path is the C-ABI library ``libadept.so`` (hand-written sm_103a CUDA);
``paper_2209_15445_gb300.adept`` is its thin ctypes binding. Importing this package
does not load the library, so the CPU-only parts (``workloads``) import anywhere.
"""
