"""GB300-native listmode SPDHG (LM-SPDHG) for sparse Poisson TOF PET data.

Submodules:
  synth  - seeded synthetic inputs (scanner, phantom, Monte Carlo events)
  lm     - binding of the C-ABI library liblmspdhg.so (CUDA, sm_103a)
"""
