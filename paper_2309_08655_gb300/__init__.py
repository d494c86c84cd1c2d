"""GB300-native batched Hamiltonian ray tracer for axion-sourced photons.

The compute path is hand-written CUDA for sm_103a behind a C ABI
(``include/rt.h``), built in place by ``paper_2309_08655_gb300.build``;
``paper_2309_08655_gb300.rt`` is a thin ctypes binding with the same names.
There is no CPU fallback: calling into the binding without the compiled
library raises.
"""
