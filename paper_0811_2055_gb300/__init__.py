"""gblod: GB300-native hierarchical level-of-detail renderer for N-body particle data.

The compute path lives in ``libgblod.so`` (hand-written sm_103a CUDA behind a C ABI); the
binding ``paper_0811_2055_gb300.gblod`` loads it and raises if it is missing.  ``synth``
generates seeded synthetic inputs.
"""
