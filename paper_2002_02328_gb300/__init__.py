"""Block 3MG (BD3MG) deblurring on one GB300: C-ABI CUDA library + thin Python binding.

Submodules:
  synth    -- seeded synthetic inputs (phantoms, PSFs, observations)
  binding  -- ctypes binding of the C-ABI library (loads the CUDA build)
  build    -- compiles the CUDA library for sm_103a
"""
__all__ = ["synth", "binding", "build"]
