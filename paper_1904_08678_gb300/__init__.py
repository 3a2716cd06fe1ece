"""GB300-native Wilson-clover multigrid (arXiv:1904.08678 hot path).

Submodules:
  build   -- compiles csrc/*.cu into libwcmg.so for sm_103a
  wcmg    -- ctypes binding of the C-ABI in include/wcmg.h (raises ImportError if not built)
  inputs  -- seeded synthetic inputs (no method arithmetic)
"""
__all__ = ["build", "wcmg", "inputs"]
