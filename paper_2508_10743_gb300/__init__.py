"""GB300-native DARC hot path (arXiv 2508.10743).

The compute path is ``libdarc.so`` (hand-written sm_103a CUDA kernels behind a
C ABI declared in ``include/darc.h``).  ``paper_2508_10743_gb300.darc`` is the
thin Python binding (argument marshalling only); ``synth`` builds seeded
synthetic cohorts; ``configs`` names the workloads.  Importing this package
does not load the CUDA library; the binding loads it on first use and raises
if it is missing.
"""
__all__ = ["configs", "synth"]
