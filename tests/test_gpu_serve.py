"""Serving on the GPU: requests of mixed scenes, sizes, sample counts and
precisions, submitted together and rendered in shared waves, give exactly the
images each gives when rendered alone, and every served image meets the
parity rule against the FP64 oracle (sampled pixels of each request)."""
import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S
from gpu_common import assert_ids, assert_rgb, id_stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0801_1500_gb300 import gbrt
    return gbrt


def test_each_result_same_alone_and_in_the_mix(G):
    import torch
    from paper_0801_1500_gb300 import serve as SV
    scenes = [S.globule(300, 285, 10.0, seed=1), S.globule(1500, 1425, 22.0, seed=2),
              S.globule(4000, 3800, 30.0, seed=3)]
    be = SV.GpuBackend(0, lam=2.0)
    srv = SV.Server(be, scenes, hbm_budget=256 << 20, wave_rays=3e6, band_rows=24)
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(14):
        si = int(rng.integers(0, 3))
        W, H = [(64, 48), (200, 150), (333, 77), (256, 256), (17, 301)][k % 5]
        spp = int([4, 16, 9][k % 3])
        prec = S.PRECISION_FP64 if k % 5 == 4 else S.PRECISION_FP32
        cam = S.ortho_camera(scenes[si], W, H, angle_deg=float(rng.uniform(0, 360)))
        reqs.append(SV.Request(scene=si, camera=cam, width=W, height=H, spp=spp, precision=prec, seed=k,
                               want_ids=True))
    futs = [srv.submit(r) for r in reqs]
    outs = [f.result(timeout=120) for f in futs]
    srv.close()
    assert srv.stats()["waves"] < len(reqs) * 4  # bands of several requests shared waves
    for k, (req, out) in enumerate(zip(reqs, outs)):
        check_against_oracle(req, out, scenes[req.scene], mode="brute", n_pix=1200, where=f"request {k}")
    with G.Renderer(0) as r:
        handles = [r.upload(sc, lam=2.0) for sc in scenes]
        for req, (rgb, ids) in zip(reqs, outs):
            sh, gh = handles[req.scene]
            p = S.Params(ao_samples=req.spp, seed=req.seed, precision=req.precision)
            ref_rgb, ref_ids, _ = r.render(sh, gh, req.camera, req.width, req.height, S.default_lights(), p,
                                           ids=True)
            G.gbrt_sync(r.ctx)
            assert torch.equal(ref_rgb, rgb) and torch.equal(ref_ids, ids)
    be.close()


def check_against_oracle(req, out, scene, mode, n_pix, where, lam=2.0):
    """Parity rule on n_pix sampled pixels of one served request."""
    import oracle
    rgb, ids = out
    n = req.width * req.height
    pix = np.random.default_rng(req.seed).choice(n, min(n, n_pix), replace=False)
    p = S.Params(ao_samples=req.spp, seed=req.seed, frame=req.frame, precision=req.precision)
    ref = oracle.render(scene, req.camera, req.width, req.height, S.default_lights(), p, pixels=pix, mode=mode,
                        lam=lam)
    got_rgb = rgb.cpu().numpy().reshape(-1, 3).astype(np.float64)[pix]
    got_ids = ids.cpu().numpy().view(np.uint32).ravel()[pix]
    assert_ids(*id_stats(got_ids, ref), len(pix), where)
    assert_rgb(np.abs(got_rgb - ref["rgb"]), where)


def test_served_images_on_the_largest_scene_match_the_oracle(G):
    # the 250k-object scene of the serving trace beside a small one, FP32 and
    # FP64 requests in one mix: every served image against the oracle
    from paper_0801_1500_gb300 import serve as SV
    big = S.globule(127500, 121125, 60.0 * (127500 / 13500.0) ** (1.0 / 3.0), seed=1)
    small = S.globule(300, 285, 10.0, seed=1)
    scenes = [small, big]
    be = SV.GpuBackend(0, lam=8.0)
    srv = SV.Server(be, scenes, hbm_budget=256 << 20, wave_rays=2e6, band_rows=32)
    specs = [(1, 256, 192, 4, S.PRECISION_FP32, 30.0), (0, 128, 96, 16, S.PRECISION_FP32, 0.0),
             (1, 160, 120, 8, S.PRECISION_FP64, 200.0), (0, 96, 64, 9, S.PRECISION_FP64, 90.0),
             (1, 200, 100, 16, S.PRECISION_FP32, 110.0)]
    reqs = [SV.Request(scene=si, camera=S.ortho_camera(scenes[si], W, H, angle_deg=ang), width=W, height=H, spp=spp,
                       precision=prec, seed=40 + k, frame=k, want_ids=True)
            for k, (si, W, H, spp, prec, ang) in enumerate(specs)]
    outs = [f.result(timeout=300) for f in [srv.submit(r) for r in reqs]]
    srv.close()
    for k, (req, out) in enumerate(zip(reqs, outs)):
        big_scene = req.scene == 1
        check_against_oracle(req, out, scenes[req.scene], mode="grid" if big_scene else "brute", n_pix=1200,
                             where=f"request {k} ({'250k' if big_scene else 'small'} scene)")
    be.close()
