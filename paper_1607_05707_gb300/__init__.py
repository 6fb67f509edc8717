"""GB300-native worklist ForAll over CSR graphs (IrGL's Iterate/Pipe/ForAll lowering).

Submodules:
  inputs  -- seeded synthetic graphs and sources (input side only)
  irgl    -- ctypes binding of the C-ABI library libirgl.so (CUDA sm_103a kernels)

Importing the package loads nothing native; ``irgl`` loads libirgl.so on first use
and raises if it is missing.
"""
__all__ = ["inputs", "irgl"]
