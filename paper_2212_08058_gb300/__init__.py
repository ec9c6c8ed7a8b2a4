"""GB300-native SFSeg / SFSeg++ power iteration (arXiv 2212.08058).

The compute path lives in the CUDA library ``libsfseg.so`` (built from ``csrc/`` for sm_103a);
``paper_2212_08058_gb300.sfseg`` is its thin Python binding.  Importing this package loads
nothing: ``synth`` (seeded input volumes) works without a GPU or the library.
"""
__all__ = ["sfseg", "synth"]
