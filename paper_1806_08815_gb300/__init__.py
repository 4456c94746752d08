"""GB300 (sm_103a) library for the Digital Annealer's parallel-trial Monte Carlo
step on dense QUBOs (Aramon et al., arXiv:1806.08815).

The compute path is the CUDA library libda.so (C ABI: include/da.h); this
package holds its ctypes binding, its build script and the seeded instance
generators.  There is no CPU fallback: without the built library or a CUDA
device the calls raise.
"""
from .binding import (DA_FP32, DA_INT8, DA_INT16, Context, DAError, da_anneal, da_anneal_async, da_anneal_plain, da_create,  # noqa: F401
                      da_destroy, da_energy, da_field_recompute, da_pt, da_set_launch_shape, da_words)

__all__ = ["DA_FP32", "DA_INT8", "DA_INT16", "Context", "DAError", "da_anneal", "da_anneal_async", "da_anneal_plain", "da_create", "da_destroy",
           "da_energy", "da_field_recompute", "da_pt", "da_set_launch_shape", "da_words"]
