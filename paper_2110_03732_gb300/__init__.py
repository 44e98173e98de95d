"""GB300-native resistive (GR)MHD IMEX stage (arXiv 2110.03732).

The compute path is the C-ABI library ``libgrmhd`` (hand-written CUDA for sm_103a,
``csrc/``); ``paper_2110_03732_gb300.grmhd`` is its thin ctypes binding.
``paper_2110_03732_gb300.problems`` holds seeded initial data only.
"""
