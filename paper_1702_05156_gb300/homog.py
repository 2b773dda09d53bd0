"""The motion-estimation front end (include/dmsgm_homog.h): the homography the
DMSGM step consumes, estimated on the GPU from two frames -- Shi-Tomasi
corners, pyramidal Lucas-Kanade, RANSAC (Sec. 2.4 and Sec. 3.1.3 of
arXiv:1702.05156).  Argument marshalling only; every step runs in the
library's CUDA kernels."""
from __future__ import annotations

import torch

from . import _lib


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _frame(f: torch.Tensor, width: int, height: int) -> int:
    if not (f.is_cuda and f.dtype == torch.uint8 and f.is_contiguous()
            and tuple(f.shape) == (height, width)):
        raise ValueError(f"frame must be a contiguous CUDA uint8 tensor of shape ({height}, {width})")
    return f.data_ptr()


class HomographyEstimator:
    """Estimates, per frame pair, H mapping current pixel centres to previous
    ones (the argument of ``Dmsgm.process``).  Keyword arguments override the
    fields of ``dmsgm_homog_params`` (block_size, quality, min_distance,
    max_corners, levels, win_half, max_iters, eps, min_eig, ransac_iters,
    thresh, seed)."""

    def __init__(self, width: int, height: int, **params):
        p = _lib.dmsgm_homog_default_params()
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.width, self.height, self.params = width, height, p
        self._h = _lib.dmsgm_homog_create(width, height, p)

    def estimate(self, prev: torch.Tensor, cur: torch.Tensor, stream=None):
        """(H as a 3x3 float64 array, result counts)."""
        return _lib.dmsgm_homog_estimate(self._h, _frame(prev, self.width, self.height),
                                         _frame(cur, self.width, self.height), _stream(stream))

    def corners(self, img: torch.Tensor, stream=None):
        """(corner pixel indices m x 2, their scores, candidates before the cap)."""
        return _lib.dmsgm_homog_corners(self._h, _frame(img, self.width, self.height),
                                        self.params.max_corners, _stream(stream))

    def track(self, prev: torch.Tensor, cur: torch.Tensor, pts, stream=None):
        """(tracked positions n x 2, status n)."""
        return _lib.dmsgm_homog_track(self._h, _frame(prev, self.width, self.height),
                                      _frame(cur, self.width, self.height), pts, _stream(stream))

    def ransac(self, src, dst, stream=None):
        """(H, inlier mask, result counts) of pairs src -> dst."""
        return _lib.dmsgm_homog_ransac(self._h, src, dst, _stream(stream))

    def close(self):
        if self._h:
            _lib.dmsgm_homog_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
