"""GB300-native VQ-NQS local-energy path (arXiv 2212.11296).

The compute runs in ``libvqnqs.so`` (hand-written sm_103a CUDA behind the C ABI
of include/vqnqs.h); this package only marshals torch device tensors and
streams into those calls.
"""
from .api import REUSE, BF16, INCREMENTAL, BF16_SPLIT, VQNQS, VQNQSError, LogPsi, LocalEnergyGraph  # noqa: F401
