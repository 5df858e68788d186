"""GB300-native decentralized coordinate-descent MIMO detection and precoding.

Implements the hot path of K. Li et al., "Decentralized Coordinate-Descent Data Detection and
Precoding for Massive MU-MIMO" (arXiv 1902.08653): per-(subcarrier, antenna-cluster) CD L-MMSE
detection (Algorithm 1) with feedforward fusion (Sec. III), and per-cluster CD ZF precoding
(Algorithm 2, Eq. (4)) with per-cluster power normalization (Sec. IV-B), as hand-written sm_103a
CUDA kernels behind the C ABI declared in include/cdmimo.h.

  cdmimo    ctypes binding of the C ABI (torch tensors in, raw pointers out)
  workload  seeded synthetic inputs (Rayleigh channels, QAM, AWGN, 16-bit storage)
  build     in-tree nvcc build of libcdmimo.so
"""
from . import workload  # noqa: F401
from .cdmimo import (CdmimoError, detect, detect_host, device_status, fuse, precode,  # noqa: F401
                     precode_host, status_string)
