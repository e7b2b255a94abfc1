"""GB300 (sm_103a) VEGAS+ iteration loop.

* ``paper_2408_09229_gb300.vegas``: Python binding of the C ABI in
  include/vegas.h (libvegas_gb300.so, hand-written CUDA kernels).
* ``paper_2408_09229_gb300.workloads``: seeded synthetic integrand parameters
  and their closed-form integrals.
"""
