"""GB300-native (sm_103a) DMSGM motion mask: motion-compensated dual-mode
single Gaussian models on a block grid (Yi et al., as restated in
arXiv:1702.05156), one fused CUDA kernel per frame behind a C ABI.

The CUDA library is loaded on first use of ``Dmsgm``; importing the package
(e.g. for ``synth``) does not need it.
"""

__all__ = ["Dmsgm", "process_batch", "mask_words", "new_mask", "unpack_mask"]


def __getattr__(name):
    if name in __all__:
        from . import dmsgm
        return getattr(dmsgm, name)
    raise AttributeError(name)
