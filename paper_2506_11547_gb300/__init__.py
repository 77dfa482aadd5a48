"""GB300-native rotation voting (arXiv 2506.11547): the data-parallel hot path
as hand-written sm_103a CUDA behind a C ABI (include/rot_vote.h).

`synth` (seeded synthetic inputs) imports without a GPU. The library binding
(`rot_vote`) loads librot_vote.so on first use and raises if it is missing:
there is no CPU fallback.
"""
__all__ = ["synth"]
