"""Shared helpers of the GPU parity tests: run a frame through the C ABI and
compare it with the FP64 oracle under the parity rule.

Parity rule (per frame):
  * hit object ids equal on every pixel the oracle marks non-grazing;
  * on grazing pixels the GPU id is the oracle's nearest, its runner-up or a miss;
  * per-channel |dRGB| <= 1/255 on at least 99.9% of pixels;
  * mean absolute error over all pixels and channels <= 1e-4.
"""
import numpy as np

RGB_TOL = 1.0 / 255.0
FRAC_OK = 0.999
MAE_TOL = 1e-4


def gpu_frame(G, r, scene, grid, cam, W, H, lights, params, spp=None):
    rgb, ids, vis = r.render(scene, grid, cam, W, H, lights, params, ao_samples=spp, ids=True, vis=True)
    G.gbrt_sync(r.ctx)
    return (rgb.cpu().numpy().reshape(-1, 3).astype(np.float64), ids.cpu().numpy().view(np.uint32).ravel(),
            vis.cpu().numpy().view(np.uint32).ravel())


def compare(rgb, ids, vis, ref, pixels=None):
    """Stats of a GPU frame (flattened) against an oracle result."""
    if pixels is not None:
        rgb, ids, vis = rgb[pixels], ids[pixels], vis[pixels]
    ok = ~ref["grazing"]
    id_mismatch = int((ids[ok] != ref["id"][ok]).sum())
    d = np.abs(rgb - ref["rgb"])
    frac_bad = float((d.max(axis=1) > RGB_TOL).mean())
    mae = float(d.mean())
    vis_eq = float((vis == ref["vis"].astype(np.uint32)).mean())
    return dict(id_mismatch=id_mismatch, n=len(ids), grazing=int((~ok).sum()), frac_bad=frac_bad, mae=mae,
                vis_eq=vis_eq, max_err=float(d.max()) if d.size else 0.0)


def assert_parity(stats, where=""):
    assert stats["id_mismatch"] == 0, (where, stats)
    assert stats["frac_bad"] <= 1.0 - FRAC_OK, (where, stats)
    assert stats["mae"] <= MAE_TOL, (where, stats)
