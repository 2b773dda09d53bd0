"""Teacher-forced comparison of one GPU frame step with the FP64 oracle.

The oracle steps from the GPU's own state at t-1 (its FP32/FP16 values are
exact in FP64), so the two sides see identical inputs and differ only by the
GPU's FP32 arithmetic.  A decision that sits within that arithmetic's reach
of its threshold may legitimately go either way; such blocks are "exempt"
from the state comparison and counted.

Bands (derived from FP32 error of one step, values <= 255 and ages <= 255):
  * compensated mean: |d mu~| <= DMU = 5e-4  (mixing of 4 neighbours in FP32
    plus the FP32 projection's weight error, ~1e-6 px at 4K)
  * compensated variance: |d var~| <= 1e-5 * var~ + 5e-4
  * a match test (M - mu~)^2 < theta_s * max(var~, 0.1) is a near tie when
    |lhs - rhs| <= 2 |M - mu~| DMU + DMU^2 + theta_s * d var~
  * a mixed age x is a near tie when |frac(x) - 1/2| <= 1e-4
  * the in-grid weight is a near tie when |W - 1e-3| <= 1e-6
Tolerances of the comparison itself:
  * ages bit-exact; mu and var within max(REL * |oracle|, 1e-5 * 255), REL =
    1e-5 for FP32 state, 6e-4 for FP16 state (half an FP16 ulp is 4.9e-4);
  * a mask pixel may differ only where |(I - mu_A)^2 - theta_d var_A| <=
    1e-4 theta_d var_A (oracle values), and at most 1e-5 of all pixels.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from oracle import DIAG, oracle_step, state_from_arrays

DMU = 5e-4
ABS_FLOOR = 1e-5 * 255


def dvar(v):
    return 1e-5 * np.abs(v) + 5e-4


@dataclass
class StepReport:
    blocks: int = 0
    exempt: int = 0
    pixels: int = 0
    mask_mismatch: int = 0
    mask_out_of_band: int = 0
    age_mismatch: int = 0
    state_out_of_tol: int = 0
    max_rel_mu: float = 0.0
    max_rel_var: float = 0.0
    max_abs_mu: float = 0.0
    max_abs_var: float = 0.0
    notes: list = field(default_factory=list)

    def add(self, o: "StepReport"):
        for k in ("blocks", "exempt", "pixels", "mask_mismatch", "mask_out_of_band",
                  "age_mismatch", "state_out_of_tol"):
            setattr(self, k, getattr(self, k) + getattr(o, k))
        for k in ("max_rel_mu", "max_rel_var", "max_abs_mu", "max_abs_var"):
            setattr(self, k, max(getattr(self, k), getattr(o, k)))
        self.notes += o.notes

    def assert_ok(self, mask_frac: float = 1e-5):
        assert self.age_mismatch == 0, self
        assert self.state_out_of_tol == 0, self
        assert self.mask_out_of_band == 0, self
        assert self.mask_mismatch <= mask_frac * max(self.pixels, 1), self


def exempt_blocks(dg: np.ndarray, theta_s: float) -> np.ndarray:
    """Blocks whose decisions sit within FP32 reach of a threshold."""
    M = dg[..., DIAG["M"]]
    src = dg[..., DIAG["NOSRC"]] == 0
    ex = np.abs(dg[..., DIAG["WSUM"]] - 1e-3) <= 1e-6
    for mu_k, var_k in (("MU_A", "VAR_A"), ("MU_C", "VAR_C")):
        mu, var = dg[..., DIAG[mu_k]], dg[..., DIAG[var_k]]
        lhs = (M - mu) ** 2
        rhs = theta_s * np.maximum(var, 0.1)
        band = 2 * np.abs(M - mu) * DMU + DMU ** 2 + theta_s * dvar(var)
        ex |= src & (np.abs(lhs - rhs) <= band)
    for x_k in ("XAGE_A", "XAGE_C"):
        x = dg[..., DIAG[x_k]]
        ex |= src & (np.abs(x - np.floor(x) - 0.5) <= 1e-4)
    return ex


def compare_step(prev: dict | None, got: dict, got_mask_bits: np.ndarray, frame: np.ndarray,
                 H: np.ndarray, *, block: int, theta_s=2.0, theta_d=4.0, age_max=30,
                 rel: float = 1e-5, mix_spread: bool = False) -> StepReport:
    """prev/got: GPU state dicts (arrays (Gy, Gx)) before/after the frame;
    prev None = first frame.  got_mask_bits: unpacked uint8 (H, W)."""
    pst = None
    if prev is not None:
        pst = state_from_arrays(*(np.asarray(prev[k], dtype=np.float64) for k in
                                  ("muA", "varA", "ageA", "muC", "varC", "ageC")))
    ost, omask, dg = oracle_step(frame, H, pst, block=block, theta_s=theta_s, theta_d=theta_d,
                                 age_max=age_max, diag=True, mix_spread=mix_spread)
    r = StepReport()
    ex = exempt_blocks(dg, theta_s)
    keep = ~ex
    r.blocks = ex.size
    r.exempt = int(ex.sum())
    for name in ("ageA", "ageC"):
        g = np.asarray(got[name]).astype(np.int64)
        o = getattr(ost, name).astype(np.int64)
        r.age_mismatch += int((g != o)[keep].sum())
    for name in ("muA", "varA", "muC", "varC"):
        g = np.asarray(got[name], dtype=np.float64)
        o = getattr(ost, name)
        err = np.abs(g - o)
        tol = np.maximum(rel * np.abs(o), ABS_FLOOR)
        bad = (err > tol) & keep
        r.state_out_of_tol += int(bad.sum())
        relerr = (err / np.maximum(np.abs(o), 1e-30))[keep]
        kind = "mu" if name.startswith("mu") else "var"
        if relerr.size:
            setattr(r, f"max_rel_{kind}", max(getattr(r, f"max_rel_{kind}"), float(relerr.max())))
            setattr(r, f"max_abs_{kind}", max(getattr(r, f"max_abs_{kind}"), float(err[keep].max())))
        if bad.any():
            idx = np.argwhere(bad)[0]
            r.notes.append(f"{name}{tuple(idx)} gpu={g[tuple(idx)]!r} oracle={o[tuple(idx)]!r}")
    # mask
    hh, ww = frame.shape   # a block row cut by the frame edge: crop the expansion
    pix_keep = np.kron(keep, np.ones((block, block), bool))[:hh, :ww]
    mism = (got_mask_bits != omask) & pix_keep
    r.pixels = int(pix_keep.sum())
    r.mask_mismatch = int(mism.sum())
    if r.mask_mismatch:
        muA = np.kron(ost.muA, np.ones((block, block)))[:hh, :ww]
        varA = np.kron(ost.varA, np.ones((block, block)))[:hh, :ww]
        f = frame.astype(np.float64)
        thr = theta_d * varA
        band = np.abs((f - muA) ** 2 - thr) <= 1e-4 * thr
        r.mask_out_of_band = int((mism & ~band).sum())
        if r.mask_out_of_band:
            idx = np.argwhere(mism & ~band)[0]
            r.notes.append(f"mask{tuple(idx)} gpu={got_mask_bits[tuple(idx)]} "
                           f"oracle={omask[tuple(idx)]} I={frame[tuple(idx)]} "
                           f"muA={muA[tuple(idx)]} varA={varA[tuple(idx)]}")
    return r
