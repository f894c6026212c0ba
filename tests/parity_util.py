"""Element-wise comparison of a GPU frame with the FP64 oracle.

A pixel matches when its unquantised RGBA is within ``tol`` (max abs per
channel) of the oracle's value -- or of the oracle's alternative value, but
only where the oracle reports that the early-termination decision sat within
``term_margin`` of the threshold (FP32 accumulation may then take the other,
equally valid side).  Pixels whose entry/exit sample decision is a near-tie
(``margin < edge_margin`` steps) or, in nearest-cell mode, whose sample lies
within ``near_margin`` voxels of a cell boundary are excluded and counted.
8-bit output must agree within 1 LSB of the matching oracle value; sample
counts must agree exactly with the matching oracle value.
"""
from __future__ import annotations

import dataclasses

import numpy as np

TOL_F32 = 1e-4        # max abs per channel before quantisation, FP32 data


@dataclasses.dataclass
class Report:
    pixels: int
    hit: int
    excluded: int
    alt_used: int
    max_err: float
    bad: int
    bad_u8: int
    bad_ns: int

    def frac_excluded(self):
        return self.excluded / max(1, self.hit)


def compare(g32, g8, gns, orc, tol=TOL_F32, term_margin=1e-3, edge_margin=1e-6,
            near_margin=1e-4, interp=1, sel=None) -> Report:
    g32 = np.asarray(g32, np.float64).reshape(-1, 4)
    g8 = np.asarray(g8).reshape(-1, 4).astype(np.int64)
    gns = np.asarray(gns).reshape(-1)
    o = {k: np.asarray(v) for k, v in orc.items()}
    if sel is not None:
        g32, g8, gns = g32[sel], g8[sel], gns[sel]
    rgba = o["rgba"].reshape(-1, 4)
    alt = o["rgba_alt"].reshape(-1, 4)
    m = o["margin"].reshape(-1, 4)
    ns, ns_alt = o["nsamp"].reshape(-1), o["nsamp_alt"].reshape(-1)
    u8, u8a = o["rgba8"].reshape(-1, 4).astype(np.int64), o["rgba8_alt"].reshape(-1, 4).astype(np.int64)

    e_main = np.abs(g32 - rgba).max(-1)
    e_alt = np.abs(g32 - alt).max(-1)
    use_alt = (e_main > tol) & (m[:, 2] < term_margin) & (e_alt <= tol)
    err = np.where(use_alt, e_alt, e_main)
    excl = (m[:, 0] < edge_margin) | (m[:, 1] < edge_margin)
    if not interp:
        excl |= m[:, 3] < near_margin
    keep = ~excl
    ref8 = np.where(use_alt[:, None], u8a, u8)
    refns = np.where(use_alt, ns_alt, ns)
    hit = int((ns > 0).sum())
    return Report(pixels=len(g32), hit=hit, excluded=int(excl.sum()), alt_used=int(use_alt.sum()),
                  max_err=float(err[keep].max()) if keep.any() else 0.0,
                  bad=int((err[keep] > tol).sum()),
                  bad_u8=int((np.abs(g8 - ref8).max(-1)[keep] > 1).sum()),
                  bad_ns=int((gns[keep] != refns[keep]).sum()))


def assert_parity(rep: Report, max_excluded_frac=1e-3, what=""):
    msg = f"{what}: {rep}"
    assert rep.bad == 0, msg
    assert rep.bad_u8 == 0, msg
    assert rep.bad_ns == 0, msg
    assert rep.frac_excluded() <= max_excluded_frac, msg
