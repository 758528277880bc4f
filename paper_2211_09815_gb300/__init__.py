"""GB300-native differentiable particle-mesh N-body with the adjoint method.

The compute path lives in the C-ABI library ``libpmgb.so`` built from ``csrc/``
(hand-written CUDA for sm_103a).  ``paper_2211_09815_gb300.pm`` is the thin ctypes
binding; it raises at first use if the library has not been built.  ``inputs`` draws
the seeded synthetic inputs and holds none of the method's arithmetic.
"""
__all__ = ["inputs", "pm", "build"]
