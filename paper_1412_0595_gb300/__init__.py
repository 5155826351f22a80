"""GB300-native time-step loop of a conductance-based Hodgkin-Huxley spiking
network with connection-density-dependent conductance scaling (Balaji,
Yavuz, Nowotny: Sec. 2 model, Sec. 3 compressed-row storage, Sec. 5.1
gScale law).

All computation runs in the CUDA library ``_build/libsnn.so`` behind the
C-ABI of ``include/snn.h``; importing this package fails if the library is
missing (there is no CPU path).  PyTorch provides device memory and streams.
"""
from ._lib import SNNError, lib  # noqa: F401  (loads the CUDA library or raises)
from .network import DenseBatch, DenseGrad, GradedNetwork, Network, SNNFunction, TorchAllocator, csr_bernoulli  # noqa: F401

__all__ = ["Network", "GradedNetwork", "SNNFunction", "DenseBatch", "DenseGrad", "TorchAllocator", "csr_bernoulli",
           "SNNError", "lib"]
