"""GB300-native catalog shift-and-stack (Stetzler et al., arXiv 2509.26279).

The hot path (project, bin, count distinct epochs, threshold, compact, order,
gather contributing ids; the candidate vetter; the batched multi-field launch)
runs in hand-written CUDA kernels for sm_103a behind the C ABI declared in
include/sas.h.  ``paper_2509_26279_gb300.sas`` is the thin ctypes binding.
"""
