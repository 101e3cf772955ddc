"""CPU oracle for the hybrid 2D/3D Gaussian rasterizer (EGGS, Sec. 3.1-3.2,
App. C-D).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import this package.  It never imports the
CUDA package (paper_2512_02932_gb300) and the CUDA package never imports it.

  native        -- ctypes front end of the FP64 C renderer (hgs_oracle.c), its
                   FP32 binning-contract replica, the SH basis and the exchange.
  autograd_ref  -- an independent FP64 torch-CPU formulation of the same
                   image function, differentiated by autograd (gradients).

Parity status of each function is recorded in its module docstring.
"""
