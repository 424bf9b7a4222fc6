"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (the sonar path's stated bar):
  - hit/miss and triangle ids identical except for rays the oracle flags as
    within 1e-6 (barycentric) of a triangle edge, as a near tie, as grazing,
    or (a cast bounded at r_max) as returning within 1e-5 relative of r_max;
  - hit range within 1e-5 relative;
  - polar bins within 1e-4 relative in FP32 (absolute floor 1e-6 of the image
    maximum), excluding the bins that receive a hit within 1e-4 m of a range
    bin edge and their neighbour across that edge.
"""
import numpy as np

NO = 0xFFFFFFFF
RTOL_R = 1e-5
RTOL_BIN = 1e-4


def gpu_hits(h):
    """Structured hit array -> (tri int64 with -1 miss, key int64 with -1, r, cos)."""
    tri = np.where(h["tri"] == NO, -1, h["tri"].astype(np.int64))
    key = np.where(h["key"] == NO, -1, h["key"].astype(np.int64))
    return tri, key, h["r"].astype(np.float64), h["cos"].astype(np.float64)


def hit_parity(ref, h, ids=None):
    """Checks per-ray results; returns the mask of rays excluded by oracle flags."""
    tri, key, r, cs = gpu_hits(h)
    if ids is not None:
        tri, key, r, cs = tri[ids], key[ids], r[ids], cs[ids]
    f = ref["flags"]
    amb = f["edge"] | f["tie"] | f["graze"] | f["limit"]
    rt = ref["hits"]["tri"].astype(np.int64)
    bad = (tri != rt) & ~amb
    assert not bad.any(), f"{bad.sum()} unflagged rays hit different triangles: {np.flatnonzero(bad)[:10]}"
    both = (tri >= 0) & (rt >= 0) & (tri == rt)
    rr = ref["hits"]["t"]
    rel = np.abs(r[both] - rr[both]) / rr[both]
    assert rel.size == 0 or rel.max() <= RTOL_R, f"range rel err {rel.max():.3g}"
    # binning: same key unless the ray is flagged
    kb = (key != ref["key"]) & ~(amb | f["binedge"])
    assert not kb.any(), f"{kb.sum()} unflagged rays binned differently: {np.flatnonzero(kb)[:10]}"
    # incidence factor
    cref = np.abs(ref["hits"]["dn"])
    ok = both & ~amb
    assert np.allclose(cs[ok], cref[ok], rtol=1e-4, atol=1e-6)
    return amb | f["binedge"]


def excluded_bins(spec, ref, h):
    """Bin mask [nr, naz] of bins a polar comparison must skip."""
    nr, naz = spec.n_range_bins, spec.n_az_bins
    _, key, _, _ = gpu_hits(h)
    f = ref["flags"]
    bad = f["edge"] | f["tie"] | f["graze"] | f["limit"] | f["binedge"] | (key != ref["key"])
    mask = np.zeros(nr * naz, bool)
    for k in np.flatnonzero(bad):
        for kk in (key[k], ref["key"][k]):
            if kk >= 0:
                mask[kk] = True
                if kk - naz >= 0:
                    mask[kk - naz] = True
                if kk + naz < nr * naz:
                    mask[kk + naz] = True
    return mask.reshape(nr, naz)


def assert_bins_close(gpu, ref, mask, rtol=RTOL_BIN, what="bins"):
    g = np.asarray(gpu, np.float64)
    r = np.asarray(ref, np.float64)
    floor = 1e-6 * max(np.abs(r).max(), 1e-30)
    ok = ~mask
    err = np.abs(g - r)
    lim = rtol * np.abs(r) + floor
    viol = ok & (err > lim)
    assert not viol.any(), (f"{what}: {viol.sum()} of {ok.sum()} bins out of tolerance; worst rel "
                            f"{(err[ok] / np.maximum(np.abs(r[ok]), floor)).max():.3g}")
