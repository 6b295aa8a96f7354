"""GB300 (sm_103a) SegSALSA-STR: the per-iteration SALSA/ADMM sweep of Condessa,
Bioucas-Dias and Kovacevic (arXiv 1504.07028) as CUDA kernels behind a C ABI
(include/segsalsa_str.h). ``binding`` loads the shared library; ``synth`` draws the seeded
synthetic scenes. Importing the package loads nothing."""
