"""GB300-native time-domain Teukolsky solver (two-step Lax-Wendroff, arXiv:1206.0270).

The compute path is the C-ABI library ``libteuk.so`` built from ``csrc/``;
``teuk`` is its thin Python binding.  ``inputs`` holds the seeded synthetic
inputs.  Submodules are imported on demand.
"""
__all__ = ["inputs", "teuk"]
