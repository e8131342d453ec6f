"""GB300 (sm_103a) SINR evaluation from the groupwise Tucker form of MIMO
channel submatrices (arXiv 2401.09792).

The compute path is the CUDA library ``libtuckersinr.so`` (C ABI:
``include/tuckersinr.h``); ``tuckersinr`` binds it with the same names;
``synth`` draws the seeded synthetic inputs; ``build`` compiles the library.
"""
