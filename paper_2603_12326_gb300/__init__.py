"""GB300 (sm_103a) all-electron RPA screening: pair densities, chi0 on tcgen05
tensor cores, batched dielectric inverse, loss functions and the halo rate,
behind the C ABI of libqcx (include/qcx.h).  ``qcx`` is the thin ctypes
binding; every step of the path runs in the library's CUDA kernels."""
from . import qcx  # noqa: F401
from .qcx import (QCX_FP64, QCX_MIXED, Context, QcxError, halo_params, library_path,  # noqa: F401
                  load)
