"""GB300 (sm_103a) library for algebraic flux correction of P1/Q1 finite element
discretisations of 3D convection-diffusion-reaction equations.

The compute path is libafc.so (CUDA, C ABI in include/afc.h); ``afc`` is its
ctypes binding and ``workloads`` builds seeded synthetic inputs."""
__all__ = ["afc", "workloads"]
