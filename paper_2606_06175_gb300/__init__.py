"""GB300 (sm_103a) implementation of the AKRA 3.0 hot path: the matrix-free normal-equation
operator H = A^T N^-1 A (+ λ_eff I) for spin-2 weak-lensing mass mapping and the CG solve
built on it.  The compute runs in libakra.so (CUDA C++, C ABI in include/akra.h); this
package is its Python binding (``akra``) and a torch.autograd wrapper (``autograd``)."""
from . import akra  # noqa: F401  (binding only; the library loads on first use)
