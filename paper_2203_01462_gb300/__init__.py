"""GB300-native FDTD + Drude adjoint topology-optimization hot path.

The compute path lives in ``libfdtd_gb300.so`` (hand-written sm_103a CUDA
behind the C ABI declared in ``include/fdtd.h``).  ``binding`` marshals
arguments to it, ``autograd`` wraps it as a ``torch.autograd.Function``, and
``inputs`` holds the seeded synthetic workloads.  Importing the package loads
nothing; the library is opened on first use and a missing build raises.
"""

__all__ = ["inputs", "binding", "autograd"]
