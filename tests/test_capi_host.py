"""Host-side checks of the C ABI (no GPU): the library loads, exports every
entry point include/gbrt.h declares, its structs match the ctypes mirrors byte
for byte, and argument validation answers without touching a device."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbrt.h")


@pytest.fixture(scope="module")
def G():
    from paper_0801_1500_gb300 import build
    build.build()
    from paper_0801_1500_gb300 import gbrt
    return gbrt


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"GBRT_API\s+[\w\s\*]*?\b(gbrt_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(G):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(G.lib, n), n
    from paper_0801_1500_gb300 import build
    for lib in (G.LIB_PATH, build.LIB, build.LIB_CHECKED):   # the checked build exports the same ABI
        out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
        exported = set(re.findall(r"\bT (gbrt_\w+)", out))
        assert set(names) == exported, lib


def test_version_and_errors(G):
    text = open(HEADER).read()
    assert G.gbrt_version() == int(re.search(r"#define GBRT_VERSION (\d+)", text).group(1))
    codes = {k: int(v) for k, v in re.findall(r"#define GBRT_(E\w+|OK) \(?(-?\d+)\)?", text)}
    assert codes == {"OK": G.OK, "EINVAL": G.EINVAL, "ENOMEM": G.ENOMEM, "EDEVICE": G.EDEVICE,
                     "ETIMEDOUT": G.ETIMEDOUT, "ETRAVERSAL": G.ETRAVERSAL, "ECAPACITY": G.ECAPACITY,
                     "EBOUNDS": G.EBOUNDS}
    for code in codes.values():
        assert G.strerror(code) and G.strerror(code) != "unknown error"
    assert G.strerror(-99) == "unknown error"
    assert G.PROFILE_ALL == int(re.search(r"#define GBRT_PROFILE_ALL (\d+)", text).group(1))
    assert G.PROFILE_AO_WALK == int(re.search(r"#define GBRT_PROFILE_AO_WALK (\d+)", text).group(1))


def test_struct_layout_matches_header(G):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "gbrt.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("gbrt_camera %zu\n", sizeof(gbrt_camera));
  printf("gbrt_lights %zu\n", sizeof(gbrt_lights));
  printf("gbrt_params %zu\n", sizeof(gbrt_params));
  printf("gbrt_render_item %zu\n", sizeof(gbrt_render_item));
  printf("gbrt_tuning %zu\n", sizeof(gbrt_tuning));
  P(gbrt_camera, half_h) P(gbrt_lights, scale) P(gbrt_params, seed) P(gbrt_params, background)
  P(gbrt_render_item, lights) P(gbrt_render_item, params) P(gbrt_render_item, out_ao_visible)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        got = dict(line.rsplit(" ", 1) for line in subprocess.run([exe], capture_output=True, text=True,
                                                                  check=True).stdout.split("\n") if line)
    mirror = {"gbrt_camera": G.gbrt_camera, "gbrt_lights": G.gbrt_lights, "gbrt_params": G.gbrt_params,
              "gbrt_render_item": G.gbrt_render_item, "gbrt_tuning": G.gbrt_tuning}
    for k, v in got.items():
        if "." in k:
            t, f = k.split(".")
            assert getattr(mirror[t], f).offset == int(v), k
        else:
            assert C.sizeof(mirror[k]) == int(v), k


def test_null_handles_rejected_without_device(G):
    assert G.lib.gbrt_sync(None) == G.EINVAL
    assert G.lib.gbrt_destroy(None) == G.OK
    assert G.lib.gbrt_scene_upload(None, None, 0, None, 0, None, None, 0, 0, None) == G.EINVAL
    assert G.lib.gbrt_grid_build(None, None, 1.0, None) == G.EINVAL
    assert G.lib.gbrt_render(None, None, None, None, 1, 1, 1, None, None, None, None, None) == G.EINVAL
    assert G.lib.gbrt_render_batch(None, None, 0, 0) == G.EINVAL
    assert G.lib.gbrt_launch_count(None) == -1
    t = G.gbrt_tuning()
    assert G.lib.gbrt_set_tuning(None, C.byref(t)) == G.EINVAL


def test_create_without_device_reports_edevice(G):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = C.c_void_p()
    assert G.lib.gbrt_create(C.byref(h), 0, None) == G.EDEVICE


def test_binding_checks_buffers_before_the_call(G):
    # the binding passes only dense buffers of the right memory kind and size
    import numpy as np
    import torch
    a = np.zeros((4, 3), np.float32)
    assert G._buf(a, 48, True, "t") == a.ctypes.data
    assert G._buf(None, 48, True, "t") is None and G._buf(1234, 48, True, "t") == 1234
    for bad, host in ((a, False),                       # numpy arrays are host memory
                      (a[:, :2], True),                 # not dense
                      (np.zeros(11, np.float32), True),  # 44 bytes < 48
                      (torch.zeros(12), False),         # a CPU tensor where device memory is expected
                      (torch.zeros(4, 3).t(), True)):   # not contiguous
        with pytest.raises(G.GbrtError) as e:
            G._buf(bad, 48, host, "t")
        assert e.value.code == G.EINVAL
    t = torch.zeros(12)
    assert G._buf(t, 48, True, "t") == t.data_ptr()   # a CPU tensor is host memory
    cam = G.make_camera(type("Cam", (), dict(kind=0, aa=2, eye=(0, 0, 1), dir=(0, 0, -1), up=(0, 1, 0),
                                              right=(1, 0, 0), half_w=1.0, half_h=1.0))())
    p = G.gbrt_params()
    p.precision = G.FP64
    assert G._frame_bytes(cam, 5, 3, p) == (5 * 3 * 3 * 8, 5 * 3 * 4 * 4)
    p.precision = G.FP32
    assert G._frame_bytes(cam, -5, 3, p) == (0, 0)
