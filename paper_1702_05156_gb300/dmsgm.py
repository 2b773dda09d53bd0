"""Pythonic wrapper of the C ABI: a handle per video stream.

``Dmsgm(W, H, block).process(frame, H3x3)`` runs one frame of the fused
motion-compensated dual-mode SGM step on the GPU and returns the bit-packed
foreground mask.  Tensors are only containers here; all the work happens in
libdmsgm.so.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (DMSGM_KERNEL_AUTO, DMSGM_KERNEL_TILE, DMSGM_STATE_FP16,
                   DMSGM_STATE_FP32)


def mask_words(width: int) -> int:
    """uint32 words per mask row."""
    return (width + 31) // 32


def new_mask(height: int, width: int, device="cuda", n: int | None = None) -> torch.Tensor:
    shape = (height, mask_words(width)) if n is None else (n, height, mask_words(width))
    return torch.zeros(shape, dtype=torch.int32, device=device)


def unpack_mask(words, width: int) -> np.ndarray:
    """Bit-packed mask (..., H, ceil(W/32)) -> uint8 (..., H, W), 1 = foreground.
    Bit j of word i is pixel 32*i + j (LSB first)."""
    if isinstance(words, torch.Tensor):
        words = words.detach().cpu().numpy()
    w = np.ascontiguousarray(words).astype(np.uint32, copy=False)
    bits = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    return bits[..., :width]


def _stream_handle(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class Dmsgm:
    """One video stream's model state on the current CUDA device."""

    def __init__(self, width: int, height: int, block: int = 4, theta_s: float = 2.0,
                 theta_d: float = 4.0, age_max: int = 30, precision: str = "fp32",
                 tile_rows: int = 0, use_pdl: bool = False, state_mem: torch.Tensor | None = None,
                 seq_tile_rows: int = 0, kernel: str = "auto", mix_spread: bool = False,
                 prefilter: tuple | None = None, prefilter_separate: bool = False,
                 checked: bool = False):
        prec = {"fp32": DMSGM_STATE_FP32, "fp16": DMSGM_STATE_FP16}[precision]
        opts = _lib.dmsgm_opts()
        opts.precision = prec
        opts.tile_rows = tile_rows
        opts.use_pdl = 1 if use_pdl else 0
        opts.seq_tile_rows = seq_tile_rows
        opts.kernel = {"auto": DMSGM_KERNEL_AUTO, "tile": DMSGM_KERNEL_TILE}[kernel]
        opts.mix_spread = 1 if mix_spread else 0
        opts.checked = 1 if checked else 0
        if prefilter is not None:   # (gauss_size, sigma, median): Sec. 2.1 preprocessing
            opts.pre_gauss, opts.pre_sigma, opts.pre_median = (int(prefilter[0]),
                                                               float(prefilter[1]),
                                                               1 if prefilter[2] else 0)
            opts.pre_separate = 1 if prefilter_separate else 0
        self._state_mem = state_mem
        if state_mem is not None:
            opts.state_mem = state_mem.data_ptr()
            opts.state_bytes = state_mem.numel() * state_mem.element_size()
        self.width, self.height, self.block = width, height, block
        self.precision = precision
        self._h = _lib.dmsgm_create(width, height, block, theta_s, theta_d, age_max, opts)
        info = self.info()
        self.grid_w, self.grid_h = info.grid_w, info.grid_h

    # ------------------------------------------------------------------ frames
    def process(self, frame: torch.Tensor, H, mask: torch.Tensor | None = None, stream=None):
        """Enqueue one frame (uint8 (H, W) on the GPU); returns the int32 mask
        tensor (H, ceil(W/32)) the kernel writes."""
        assert frame.dtype == torch.uint8 and frame.is_cuda and frame.is_contiguous()
        assert tuple(frame.shape) == (self.height, self.width)
        if mask is None:
            mask = new_mask(self.height, self.width, frame.device)
        assert mask.is_cuda and mask.dtype == torch.int32 and mask.is_contiguous()
        assert tuple(mask.shape) == (self.height, mask_words(self.width))
        _lib.dmsgm_process(self._h, frame.data_ptr(), H, mask.data_ptr(), _stream_handle(stream))
        return mask

    def process_seq(self, frames: torch.Tensor, Hs, masks: torch.Tensor | None = None,
                    stream=None):
        """Enqueue n consecutive frames (uint8 (n, H, W) on the GPU) in
        persistent multi-frame launches; returns the masks (n, H, ceil(W/32))."""
        assert frames.dtype == torch.uint8 and frames.is_cuda and frames.is_contiguous()
        n = frames.shape[0]
        assert tuple(frames.shape[1:]) == (self.height, self.width)
        if masks is None:
            masks = new_mask(self.height, self.width, frames.device, n=n)
        assert masks.is_cuda and masks.dtype == torch.int32 and masks.is_contiguous()
        assert tuple(masks.shape) == (n, self.height, mask_words(self.width))
        _lib.dmsgm_process_seq(self._h, frames.data_ptr(), n, np.asarray(Hs), masks.data_ptr(),
                               _stream_handle(stream))
        return masks

    def process_host(self, frames: torch.Tensor, Hs, masks: torch.Tensor | None = None,
                     stream=None):
        """Enqueue n frames from host memory (uint8 (n, H, W), pinned for
        overlap) into host masks (int32 (n, H, ceil(W/32)))."""
        assert frames.dtype == torch.uint8 and not frames.is_cuda and frames.is_contiguous()
        n = frames.shape[0]
        if masks is None:
            masks = torch.zeros((n, self.height, mask_words(self.width)), dtype=torch.int32,
                                pin_memory=True)
        assert not masks.is_cuda and masks.is_contiguous()
        _lib.dmsgm_process_host(self._h, frames.data_ptr(), n, np.asarray(Hs),
                                masks.data_ptr(), _stream_handle(stream))
        return masks

    # ------------------------------------------------------------------ state
    def _layout(self):
        n = self.grid_w * self.grid_h
        fdt = np.float16 if self.precision == "fp16" else np.float32
        return n, fdt

    def get_state(self) -> dict:
        """Current state as arrays of shape (grid_h, grid_w) (synchronises).
        The packed image holds mu (A, C pairs), var (A, C pairs), age (A, C
        byte pairs), block by block."""
        n, fdt = self._layout()
        buf = np.zeros(self.info().host_state_bytes, dtype=np.uint8)
        _lib.dmsgm_get_state(self._h, buf)
        fs = np.dtype(fdt).itemsize
        shp = (self.grid_h, self.grid_w)
        mu = buf[:2 * n * fs].view(fdt).reshape(n, 2)
        var = buf[2 * n * fs:4 * n * fs].view(fdt).reshape(n, 2)
        age = buf[4 * n * fs:4 * n * fs + 2 * n].reshape(n, 2)
        return {"muA": mu[:, 0].reshape(shp).copy(), "muC": mu[:, 1].reshape(shp).copy(),
                "varA": var[:, 0].reshape(shp).copy(), "varC": var[:, 1].reshape(shp).copy(),
                "ageA": age[:, 0].reshape(shp).copy(), "ageC": age[:, 1].reshape(shp).copy()}

    def set_state(self, st: dict):
        n, fdt = self._layout()
        pair = lambda a, c, dt: np.stack(  # noqa: E731
            [np.asarray(st[a], dtype=dt).reshape(-1), np.asarray(st[c], dtype=dt).reshape(-1)],
            axis=1)
        parts = [pair("muA", "muC", fdt), pair("varA", "varC", fdt),
                 pair("ageA", "ageC", np.uint8)]
        buf = np.concatenate([np.ascontiguousarray(p).view(np.uint8).reshape(-1) for p in parts])
        assert buf.size == self.info().host_state_bytes
        _lib.dmsgm_set_state(self._h, buf)

    def reset(self):
        _lib.dmsgm_reset(self._h)

    def info(self) -> _lib.dmsgm_info:
        return _lib.dmsgm_get_info(self._h)

    def status(self) -> int:
        return _lib.dmsgm_status(self._h)

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.dmsgm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prefilter(frame: torch.Tensor, gauss_size: int = 5, sigma: float = 1.0, median: bool = True,
              out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The paper's preprocessing (Sec. 2.1) of one uint8 (H, W) CUDA frame:
    N x N Gaussian blur (gauss_size 0: none), then the 3 x 3 median."""
    assert frame.dtype == torch.uint8 and frame.is_cuda and frame.is_contiguous()
    H, W = frame.shape
    if out is None:
        out = torch.empty_like(frame)
    _lib.dmsgm_prefilter(frame.data_ptr(), out.data_ptr(), W, H, gauss_size, sigma,
                         1 if median else 0, _stream_handle(stream))
    return out


def process_batch(models, frames, Hs, masks, stream=None, ctas: int = 0, use_pdl: bool = False,
                  item_warps: int = 0):
    """One frame for each of several handles in one batched launch
    (dmsgm_batch_opts: ctas, use_pdl, item_warps)."""
    opts = _lib.dmsgm_batch_opts(0, ctas, 1 if use_pdl else 0, item_warps)
    _lib.dmsgm_process_batch([m.handle for m in models], [f.data_ptr() for f in frames],
                             np.asarray(Hs), [k.data_ptr() for k in masks],
                             _stream_handle(stream), opts)
