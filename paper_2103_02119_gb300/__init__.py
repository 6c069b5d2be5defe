"""GB300-native rectangular central-moment lattice Boltzmann method (RC-LBM).

The compute path is the C-ABI library ``liblbm_gb300.so`` (hand-written CUDA
for sm_103a, declared in ``include/lbm.h``); ``paper_2103_02119_gb300.lbm`` is
its thin ctypes binding.  Importing the binding fails loudly when the library
has not been built: there is no CPU fallback.

``paper_2103_02119_gb300.workloads`` holds the seeded synthetic inputs.
"""
__all__ = ["lbm", "workloads"]
