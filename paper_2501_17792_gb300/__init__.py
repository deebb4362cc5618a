"""GB300-native CrowdSplat crowd-synthesis path (LBS of shared template
Gaussians, distance LoD, EWA projection with SH colour, tile binning with a
(tile, depth) radix sort, front-to-back alpha compositing).

The compute path is the CUDA library ``libcrowdsplat.so`` built from
``csrc/`` for sm_103a; ``binding`` is a thin ctypes layer over its C ABI.
``scene`` draws seeded synthetic crowds.  Importing this package loads
nothing; ``binding.load()`` loads the library and raises if it is missing.
"""
__all__ = ["scene", "binding"]
