"""GB300-native fast aperture-mass maps (Leonard, Pires & Starck 2012).

The compute lives in the C-ABI library ``libfastmap.so`` (hand-written CUDA
for sm_103a).  ``paper_1204_4293_gb300.fastmap`` is its thin Python binding;
``paper_1204_4293_gb300.synth`` draws seeded synthetic inputs.  Importing this
package does not load the library; importing ``fastmap`` does, and fails
loudly if it is missing.
"""
__all__ = ["fastmap", "synth"]
