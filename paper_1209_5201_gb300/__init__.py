"""GB300 (sm_103a) streaming-collision lattice Boltzmann library with the
kinetic diffuse-reflection wall of Meng & Zhang (arXiv:1209.5201).

The compute path is the in-tree CUDA library (csrc/, built by build.py into
_build/liblbm_gb300.so); lbm.py is its ctypes binding.
"""
