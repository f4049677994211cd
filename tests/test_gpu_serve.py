"""Serving on the GPU: requests of mixed scenes, sizes, sample counts and
precisions, submitted together and rendered in shared waves, give exactly the
images each gives when rendered alone."""
import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S

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
