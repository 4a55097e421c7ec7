"""Stolt-based apex-shifted hyperbolic Radon transform (ASHRT/AASHRT) and
robust IRLS deblending on NVIDIA GB300 (sm_103a).

The compute path is the C-ABI library ``libashrt.so`` built from ``csrc/``;
``ashrt`` is its thin ctypes binding (argument marshalling only).  ``synth``
holds the seeded synthetic gather generator used by tests and the bench.
"""
