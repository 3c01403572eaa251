"""GB300-native sparse Sinkhorn-Knopp Word Mover's Distance.

The compute path is the CUDA library in ``csrc/`` behind the C ABI declared in
``include/wmd.h``; ``paper_2005_06727_gb300.wmd`` is its thin Python binding
(argument marshalling only).  ``synth`` draws seeded synthetic inputs.
"""
__all__ = ["wmd", "synth"]
