"""GB300 (sm_103a) deflated shifted block CG (DSBlockCG) for Wilson fermions.

  paper_1205_0359_gb300.dsbcg  -- ctypes binding of libdsbcg.so (C ABI in include/dsbcg.h)
  paper_1205_0359_gb300.synth  -- seeded synthetic inputs (links, right-hand sides, shifts)
  paper_1205_0359_gb300.build  -- builds libdsbcg.so in-tree with nvcc for sm_103a
"""
__all__ = ["dsbcg", "synth", "build"]
