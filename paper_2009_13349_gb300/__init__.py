"""GB300-native batched inclusion-based CCD root finder (Wang et al., Sec. 4).

The compute path is the C-ABI CUDA library built from ``csrc/``; the Python
binding in ``ccd.py`` only marshals arguments to it.  ``workloads.py`` holds
the seeded synthetic input generators.
"""
