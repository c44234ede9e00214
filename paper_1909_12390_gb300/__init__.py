"""GB300 (sm_103a) implementation of the time step of the thermodynamically consistent
multi-component pseudo-potential lattice Boltzmann model of Peng, Ayala & Ayala
(arXiv:1909.12390), behind the C ABI of include/lbm.h."""
from .lbm import (BGK, D2Q9, D3Q19, FP32_SHIFTED, FP64, MRT, LBMError, Lattice,  # noqa: F401
                  scale_to_lattice)
