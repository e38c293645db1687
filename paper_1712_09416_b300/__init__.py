"""B300-native TPC sector tracker: cellular-automaton track finding and Kalman fit.

The compute path lives in the CUDA library ``libtpctrack.so`` (``csrc/``) behind
the C ABI declared in ``include/tpctrack.h``; ``tpctrack`` is its thin ctypes
binding.  ``synth`` generates the seeded synthetic events.  Submodules are
imported on demand so that the event generator needs neither CUDA nor the
library.
"""
__all__ = ["synth", "tpctrack"]
