"""Seeded random sweep of the render's options through the C ABI against the
FP64 oracle's brute-force definition: scene size and shape, grid density,
orthographic or pinhole camera and its angle, ragged frame sizes, AO sample
counts (0 included), direct-light shadows, supersampling and precision. Each
configuration meets the parity rule: hit ids exact off grazing sub-samples,
|dRGB| <= 1/255 on all but 0.1% of pixels (at least one pixel allowed on tiny
frames), mean absolute error <= 1e-4."""
import dataclasses

import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S
from gpu_common import assert_ids, assert_rgb, id_stats

pytestmark = pytest.mark.gpu

N_CONFIGS = 64


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0801_1500_gb300 import gbrt
    return gbrt


@pytest.fixture(scope="module")
def R(G):
    r = G.Renderer(0)
    yield r
    r.close()


def config(k):
    rng = np.random.default_rng(1000 + k)
    n_s = int(rng.integers(20, 700))
    n_c = int(rng.integers(0, n_s))
    radius = float(4.0 + 0.03 * n_s)
    sc = S.globule(n_s, n_c, radius, seed=k)
    W, H = int(rng.integers(1, 90)), int(rng.integers(1, 70))
    angle = float(rng.uniform(0.0, 360.0))
    aa = int(rng.choice([1, 1, 2, 3]))
    if rng.random() < 0.5:
        cam = dataclasses.replace(S.ortho_camera(sc, W, H, angle_deg=angle), aa=aa)
    else:
        cam = S.pinhole_camera(sc, W, H, angle_deg=angle, fov_deg=float(rng.uniform(20.0, 60.0)), aa=aa)
    p = S.Params(ao_samples=int(rng.integers(0, 13)), seed=int(rng.integers(0, 2 ** 40)),
                 frame=int(rng.integers(0, 1000)),
                 precision=S.PRECISION_FP64 if rng.random() < 0.3 else S.PRECISION_FP32,
                 shadows=bool(rng.random() < 0.4))
    lam = float(rng.choice([0.5, 1.0, 2.0, 4.0, 8.0]))
    return sc, cam, W, H, p, lam


@pytest.mark.parametrize("k", range(N_CONFIGS))
def test_random_configuration_vs_brute_force(G, R, oracle, k):
    sc, cam, W, H, p, lam = config(k)
    lights = S.default_lights()
    scene, grid = R.upload(sc, lam=lam)
    rgb, ids, vis = R.render(scene, grid, cam, W, H, lights, p, ids=True, vis=True)
    G.gbrt_sync(R.ctx)
    ref = oracle.render(sc, cam, W, H, lights, p, mode="brute")
    m = cam.aa
    # per sub-sample ids and AO counts: the finer raster [m H][m W] against the
    # oracle's pixel-major, sub-row, sub-column order
    fine_ids = ids.cpu().numpy().view(np.uint32).reshape(m * H, m * W)
    fine_vis = vis.cpu().numpy().view(np.uint32).reshape(m * H, m * W)
    got_ids = fine_ids.reshape(H, m, W, m).transpose(0, 2, 1, 3).ravel()
    got_vis = fine_vis.reshape(H, m, W, m).transpose(0, 2, 1, 3).ravel()
    assert_ids(*id_stats(got_ids, ref), len(got_ids), (k, W, H, m, p))
    assert_rgb(np.abs(rgb.cpu().numpy().reshape(-1, 3).astype(np.float64) - ref["rgb"]), (k, W, H, m, p))
    if p.precision == S.PRECISION_FP64:
        assert float((got_vis == ref["vis"].astype(np.uint32)).mean()) >= 0.99, k
    R.free(scene, grid)
