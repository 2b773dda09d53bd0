"""Seeded synthetic video for the DMSGM motion mask.

This module makes INPUTS only (frames and the exact per-frame homography); it
holds none of the method's arithmetic, so both the CUDA path and the oracle
can be fed from it.

Recipe (the paper evaluates on CDNet sequences, which are not available here;
these streams stand in for them with the same shape -- 320x240 uint8 grey in
the paper's timing runs):

* background canvas: U(0, 255) noise blurred by a Gaussian of sigma 3 px
  (reflect border), larger than the frame by a margin that covers the
  largest camera displacement plus 8 px;
* camera: frame t samples the canvas bilinearly through a similarity pose
  P_t about the frame centre -- rotation U(+-0.5 deg), translation
  U(+-3 px) per axis, scale 1 + U(+-0.5 %), all multiplied by ``jitter``;
  poses jitter about a fixed pose (no random walk);
* the homography handed to the method with frame t is
  H_t = P_{t-1}^{-1} o P_t, mapping CURRENT pixel-centre coordinates to
  PREVIOUS ones, exactly (FP64); frame 0 gets the identity;
* objects: ``n_objects`` axis-aligned rectangles, sides U(W/20, W/6),
  constant intensity U(0, 255), speed U(1, 4) px/frame in a random
  direction, bouncing at the canvas edge, drawn on the canvas after the
  background;
* sensor noise N(0, 3) per pixel, rounded half to even, clipped to [0, 255].

Scalar draws (poses, objects) come from ``numpy.random.Generator(PCG64(seed))``
and are device independent; the per-pixel fields (canvas noise, sensor noise)
come from a ``torch.Generator`` seeded with ``seed`` on the target device, so
a stream is a deterministic function of (spec, device type).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch
import torch.nn.functional as F


@dataclass(frozen=True)
class StreamSpec:
    width: int
    height: int
    frames: int
    n_objects: int = 3
    jitter: float = 1.0
    seed: int = 0
    blur_sigma: float = 3.0
    noise_sigma: float = 3.0


def spec_for(width: int, height: int, frames: int, seed: int) -> StreamSpec:
    """Stream settings by resolution: up to 640 px wide, 3 objects and base
    camera jitter; wider frames, 12 objects and doubled jitter (the 1920x1080
    recipe)."""
    small = width <= 640
    return StreamSpec(width, height, frames, n_objects=3 if small else 12,
                      jitter=1.0 if small else 2.0, seed=seed)


def _pose(theta: float, s: float, tx: float, ty: float, cx: float, cy: float) -> np.ndarray:
    """Similarity about (cx, cy): x -> R(theta) * s * (x - c) + c + t."""
    c, sn = math.cos(theta) * s, math.sin(theta) * s
    A = np.array([[c, -sn], [sn, c]], dtype=np.float64)
    ctr = np.array([cx, cy], dtype=np.float64)
    off = ctr - A @ ctr + np.array([tx, ty], dtype=np.float64)
    P = np.eye(3, dtype=np.float64)
    P[:2, :2] = A
    P[:2, 2] = off
    return P


def _gauss_blur(img: torch.Tensor, sigma: float) -> torch.Tensor:
    r = int(math.ceil(3 * sigma))
    x = torch.arange(-r, r + 1, dtype=torch.float64, device=img.device)
    k = torch.exp(-0.5 * (x / sigma) ** 2)
    k = k / k.sum()
    t = img[None, None]
    t = F.pad(t, (r, r, 0, 0), mode="reflect")
    t = F.conv2d(t, k.view(1, 1, 1, -1))
    t = F.pad(t, (0, 0, r, r), mode="reflect")
    t = F.conv2d(t, k.view(1, 1, -1, 1))
    return t[0, 0]


def make_stream(spec: StreamSpec, device: str | torch.device = "cpu"):
    """Return ``(frames, Hs)``: uint8 tensor (T, H, W) on ``device`` and a
    float64 NumPy array (T, 3, 3) of current->previous homographies."""
    W, Hh, T = spec.width, spec.height, spec.frames
    dev = torch.device(device)
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    tg = torch.Generator(device=dev)
    tg.manual_seed(int(spec.seed))

    j = spec.jitter
    max_rot = math.radians(0.5 * j)
    max_t = 3.0 * j
    max_s = 0.005 * j
    # largest displacement of any frame point under a pose: rotation and
    # scale about the centre plus the translation
    half_diag = 0.5 * math.hypot(W, Hh)
    reach = half_diag * (abs(max_rot) + max_s) * 1.05 + max_t * math.sqrt(2)
    margin = int(math.ceil(reach)) + 8
    CW, CH = W + 2 * margin, Hh + 2 * margin

    bg = torch.rand((CH, CW), generator=tg, device=dev, dtype=torch.float64) * 255.0
    bg = _gauss_blur(bg, spec.blur_sigma)

    cx, cy = 0.5 * W, 0.5 * Hh
    poses = []
    for _ in range(T):
        th = rng.uniform(-max_rot, max_rot)
        tx = rng.uniform(-max_t, max_t)
        ty = rng.uniform(-max_t, max_t)
        s = 1.0 + rng.uniform(-max_s, max_s)
        poses.append(_pose(th, s, tx, ty, cx, cy))

    objs = []
    for _ in range(spec.n_objects):
        ow = rng.uniform(W / 20.0, W / 6.0)
        oh = rng.uniform(W / 20.0, W / 6.0)
        ox = rng.uniform(0.0, CW - ow)
        oy = rng.uniform(0.0, CH - oh)
        val = rng.uniform(0.0, 255.0)
        spd = rng.uniform(1.0, 4.0)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        objs.append([ox, oy, ow, oh, val, spd * math.cos(ang), spd * math.sin(ang)])

    ys, xs = torch.meshgrid(
        torch.arange(Hh, dtype=torch.float64, device=dev) + 0.5,
        torch.arange(W, dtype=torch.float64, device=dev) + 0.5, indexing="ij")
    frames = torch.empty((T, Hh, W), dtype=torch.uint8, device=dev)
    Hs = np.zeros((T, 3, 3), dtype=np.float64)
    for t in range(T):
        canvas = bg.clone()
        for o in objs:
            x0, y0 = int(round(o[0])), int(round(o[1]))
            x1, y1 = int(round(o[0] + o[2])), int(round(o[1] + o[3]))
            canvas[max(y0, 0):min(y1, CH), max(x0, 0):min(x1, CW)] = o[4]
        P = torch.tensor(poses[t], dtype=torch.float64, device=dev)
        # frame pixel centre -> canvas coordinates (canvas pixel centres at +0.5)
        u = P[0, 0] * xs + P[0, 1] * ys + P[0, 2] + margin - 0.5
        v = P[1, 0] * xs + P[1, 1] * ys + P[1, 2] + margin - 0.5
        u0, v0 = torch.floor(u), torch.floor(v)
        fu, fv = u - u0, v - v0
        iu = u0.long().clamp(0, CW - 2)
        iv = v0.long().clamp(0, CH - 2)
        c00 = canvas[iv, iu]
        c01 = canvas[iv, iu + 1]
        c10 = canvas[iv + 1, iu]
        c11 = canvas[iv + 1, iu + 1]
        img = (c00 * (1 - fu) * (1 - fv) + c01 * fu * (1 - fv)
               + c10 * (1 - fu) * fv + c11 * fu * fv)
        img = img + spec.noise_sigma * torch.randn(
            (Hh, W), generator=tg, device=dev, dtype=torch.float64)
        frames[t] = torch.round(img).clamp_(0, 255).to(torch.uint8)
        Hs[t] = np.eye(3) if t == 0 else np.linalg.solve(poses[t - 1], poses[t])
        for o in objs:  # move and bounce at the canvas edge
            o[0] += o[5]
            o[1] += o[6]
            if o[0] < 0 or o[0] + o[2] > CW:
                o[5] = -o[5]
                o[0] = min(max(o[0], 0.0), CW - o[2])
            if o[1] < 0 or o[1] + o[3] > CH:
                o[6] = -o[6]
                o[1] = min(max(o[1], 0.0), CH - o[3])
    return frames, Hs


def translation(dx: float, dy: float) -> np.ndarray:
    """Homography of a pure translation of the content: a point at x in the
    current frame was at x - (dx, dy) in the previous one."""
    H = np.eye(3, dtype=np.float64)
    H[0, 2] = -dx
    H[1, 2] = -dy
    return H


def random_state(gy: int, gx: int, age_max: int, seed: int):
    """A plausible random block state (FP64 means/variances, int ages) used to
    start teacher-forced comparisons from the middle of a sequence."""
    rng = np.random.Generator(np.random.PCG64(seed))
    muA = rng.uniform(0, 255, (gy, gx))
    muC = rng.uniform(0, 255, (gy, gx))
    varA = rng.uniform(0.05, 300, (gy, gx))
    varC = rng.uniform(0.05, 300, (gy, gx))
    ageA = rng.integers(1, age_max + 1, (gy, gx)).astype(np.int32)
    ageC = rng.integers(1, age_max + 1, (gy, gx)).astype(np.int32)
    return muA, varA, ageA, muC, varC, ageC
