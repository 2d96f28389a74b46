"""GB300-native fused lattice-Boltzmann time step for 3-D periodic Hall-MHD.

The method is the FLAME scheme of Foldes et al. (arXiv 2212.11024): a D3Q27
central-moment fluid (Sec. 3.1) coupled to three D3Q7 BGK magnetic
populations whose equilibrium carries the Hall term (Sec. 3.2), with the
current obtained from the magnetic non-equilibrium moments.

- ``Flame``   : ctypes binding of libflame.so (include/flame.h); CUDA only.
                The step runs one of two kernels: the row kernel (FP16/BF16
                storage: TMA-staged x rows, two sites per thread in packed
                FP32) or the one-site kernel (FP32 storage, and row lengths
                the row kernel does not take); both run every variant.
- ``inputs``  : seeded synthetic initial conditions (numpy).
- ``units``   : lattice-unit parameter mapping and the whistler CFL check.
- ``adjoint`` : gradients of a band magnetic energy through N steps
                (FlameBandEnergy autograd Function, sqrt(N) checkpointing).
- ``turbulence``: decaying-turbulence runs with spectra and step throughput.
- ``throughput``: step throughput of any variant, storage and kernel.
- ``budget``  : the wavenumber energy budget S(k), D(k) of Sec. 4.4 (torch.fft).
- ``validation``: the Table 1 three-mode runs and the paper's error metrics.
- ``build``   : nvcc build of libflame.so for sm_103a.
"""
from . import inputs, units
from .flame import Flame, FlameError, FlameUnavailable, lattice, library, make_params, state_bytes

__all__ = ["Flame", "FlameError", "FlameUnavailable", "inputs", "units", "lattice", "library", "make_params",
           "state_bytes"]
