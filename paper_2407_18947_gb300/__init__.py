"""RT-CC3 approximate-triples hot path on GB300 (sm_103a).

The compute path is ``librtcc3.so`` (CUDA kernels behind the C ABI of
``include/rtcc3.h``); this package is its thin Python binding.  Importing the
package is cheap: the shared library is loaded on first use.
"""

__all__ = ["RTCC3", "TriplesResidual", "synth"]


def __getattr__(name):
    if name == "RTCC3":
        from .api import RTCC3
        return RTCC3
    if name == "TriplesResidual":
        from .autograd import TriplesResidual
        return TriplesResidual
    raise AttributeError(name)
