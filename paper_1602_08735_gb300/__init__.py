"""GB300 (sm_103a) engine for the hybrid-P-system heuristics for the Variable
Sized Bin Packing Problem (Alenezi et al., arXiv:1602.08735).

The packing itself runs in the CUDA library ``libvsbpp.so`` (C ABI in
``include/vsbpp.h``); ``native`` is its thin ctypes binding, ``instances``
draws seeded synthetic inputs, ``build`` compiles the library for sm_103a.
Nothing is imported eagerly, so ``import paper_1602_08735_gb300`` works on a
machine without a GPU.
"""

__all__ = ["native", "instances", "build"]
