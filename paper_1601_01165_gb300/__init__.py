"""GB300-native brute-force incoherent dedispersion (Sclocco et al., Algorithm 1).

The compute runs in hand-written sm_103a CUDA kernels inside ``libdd.so``,
reached through a C ABI (``include/dd.h``).  This package is the thin Python
binding over that ABI; importing it does not load the library, the first call
that needs it does (and fails loudly if it is not built).
"""
__all__ = ["synth", "binding"]
