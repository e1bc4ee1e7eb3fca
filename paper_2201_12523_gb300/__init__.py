"""GB300-native sparse MTTKRP over a blocked, linearized coordinate store.

Submodules (imported on demand, so that importing the package costs nothing):

* ``blco``   -- the Python binding of the C-ABI library ``libblco.so``
               (argument marshalling only; every step runs in CUDA kernels).
* ``synth``  -- seeded synthetic input generators (no method arithmetic).
* ``build_lib`` -- compiles the CUDA sources into ``libblco.so`` for sm_103a.
"""

__all__ = ["blco", "synth", "build_lib"]
