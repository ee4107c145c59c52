"""GB300-native domain-wall fermion hot path: even-odd Shamir/Moebius operators,
CG on the normal equations, mixed-precision CG with reliable updates, the
Moebius-accelerated DWF solve (MADWF), the fermion force and the force-gradient
link update, all as hand-written sm_103a CUDA kernels behind a C ABI
(``include/dwf.h``).  The Python layer only marshals arguments.

Import ``paper_1111_5059_gb300.dwf`` for the binding; it loads ``libdwf.so``
and raises if the library is missing.
"""
