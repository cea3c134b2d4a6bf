"""GB300-native SMC-X swap-sweep engine (arXiv 2509.20949).

The hot path -- checkerboard link-cell Metropolis swap sweeps with EPI
energies, Warren-Cowley SRO and total-energy reductions -- runs in
libsmcx.so (CUDA kernels for sm_103a behind the C ABI of include/smcx.h).
This package only binds it: ``Lattice`` wraps one lattice.  Importing the
package does not load the library; the first ``Lattice`` does, and raises if
it cannot.
"""
from ._lib import SmcxError, build, lib  # noqa: F401

__all__ = ["Lattice", "Batch", "SmcxError", "build", "lib"]


def __getattr__(name):
    if name == "Lattice":
        from .lattice import Lattice
        return Lattice
    if name == "Batch":
        from .batch import Batch
        return Batch
    raise AttributeError(name)
