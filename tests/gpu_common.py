"""Shared helpers of the GPU parity tests: run a frame through the C ABI and
compare it with the FP64 oracle under the parity rule.

Parity rule (per frame):
  * hit object ids equal on every pixel the oracle marks non-grazing;
  * on grazing pixels the GPU id is one of the outcomes the oracle reports as
    within rounding: its nearest hit, its runner-up (second-nearest distinct
    hit), the object of its nearest grazing encounter, or a miss;
  * grazing pixels stay rare (at most 0.5% of the frame, plus 2), so the
    classifier cannot quietly shrink the set of pixels whose ids are checked;
  * per-channel |dRGB| <= 1/255 on at least 99.9% of pixels;
  * mean absolute error over all pixels and channels <= 1e-4.
"""
import numpy as np

RGB_TOL = 1.0 / 255.0
FRAC_OK = 0.999
MAE_TOL = 1e-4
MISS = 0xFFFFFFFF
GRAZE_FRAC_MAX = 0.005
GRAZE_ABS = 2


def gpu_frame(G, r, scene, grid, cam, W, H, lights, params, spp=None):
    rgb, ids, vis = r.render(scene, grid, cam, W, H, lights, params, ao_samples=spp, ids=True, vis=True)
    G.gbrt_sync(r.ctx)
    return (rgb.cpu().numpy().reshape(-1, 3).astype(np.float64), ids.cpu().numpy().view(np.uint32).ravel(),
            vis.cpu().numpy().view(np.uint32).ravel())


def id_stats(ids, ref):
    """Hit-id checks of GPU ids (one per oracle sub-sample, same order):
    mismatches on non-grazing entries, grazing entries whose id is none of
    the oracle's alternatives, and the number of grazing entries."""
    gz = ref["grazing"]
    ok = ~gz
    id_mismatch = int((ids[ok] != ref["id"][ok]).sum())
    g_ids = ids[gz]
    allowed = (g_ids == ref["id"][gz]) | (g_ids == MISS)
    for key in ("id2", "idg"):
        if key in ref:
            allowed |= g_ids == ref[key][gz]
    return id_mismatch, int((~allowed).sum()), int(gz.sum())


def compare(rgb, ids, vis, ref, pixels=None):
    """Stats of a GPU frame (flattened) against an oracle result."""
    if pixels is not None:
        rgb, ids, vis = rgb[pixels], ids[pixels], vis[pixels]
    id_mismatch, graze_bad, grazing = id_stats(ids, ref)
    d = np.abs(rgb - ref["rgb"])
    frac_bad = float((d.max(axis=1) > RGB_TOL).mean())
    mae = float(d.mean())
    vis_eq = float((vis == ref["vis"].astype(np.uint32)).mean())
    return dict(id_mismatch=id_mismatch, graze_bad=graze_bad, n=len(ids), grazing=grazing, frac_bad=frac_bad,
                mae=mae, vis_eq=vis_eq, max_err=float(d.max()) if d.size else 0.0)


def assert_ids(id_mismatch, graze_bad, grazing, n, where=""):
    assert id_mismatch == 0, (where, "non-grazing id mismatches", id_mismatch)
    assert graze_bad == 0, (where, "grazing ids outside the oracle's alternatives", graze_bad)
    assert grazing <= GRAZE_FRAC_MAX * n + GRAZE_ABS, (where, "grazing entries", grazing, n)


def assert_rgb(d, where=""):
    """Colour part of the rule on per-pixel absolute differences d [n, 3]."""
    frac_bad = float((d.max(axis=1) > RGB_TOL).mean()) if len(d) else 0.0
    mae = float(d.mean()) if d.size else 0.0
    assert frac_bad <= 1.0 - FRAC_OK, (where, "fraction beyond 1/255", frac_bad, float(d.max()))
    assert mae <= MAE_TOL, (where, "MAE", mae)


def assert_parity(stats, where=""):
    assert_ids(stats["id_mismatch"], stats["graze_bad"], stats["grazing"], stats["n"], where)
    assert stats["frac_bad"] <= 1.0 - FRAC_OK, (where, stats)
    assert stats["mae"] <= MAE_TOL, (where, stats)
