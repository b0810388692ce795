"""GB300 (sm_103a) library for fixed-step RK4 integration of coupled
Hodgkin-Huxley networks (Mohanta & Assisi, arXiv:1906.03958).

``psst``   -- binding of the C interface (include/psst.h) to the CUDA library
``netgen`` -- seeded synthetic network generators
``build``  -- nvcc build of the CUDA library
"""
