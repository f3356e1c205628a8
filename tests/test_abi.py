"""CPU-side checks of the C-ABI library: it loads, exports every entry point
include/fgl.h declares, validates arguments, and its host BVH builder makes
conservative quantized boxes (checked here independently of the library's
own verifier)."""

import ctypes
import os
import re

import numpy as np
import pytest

import synth
import paper_2509_17390_gb300 as fgl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fgl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fgl_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = fgl.lib()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert L.fgl_version() >= 100


def test_header_compiles_as_c(tmp_path):
    c = tmp_path / "t.c"
    c.write_text('#include "fgl.h"\nint main(void){return (int)FGL_OK;}\n')
    import subprocess
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(c), "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


# ---------------------------------------------------------------------------
# host builder
# ---------------------------------------------------------------------------
def decode_nodes(nodes: np.ndarray, width: int):
    """Node records as laid out by the builder: width 8 in 112 B (hit bits at
    80, quantized planes at 32), width 4 in 64 B (hit bits at 24, planes at 40)."""
    S, HB, Q = (112, 80, 32) if width == 8 else (64, 24, 40)
    rec = nodes.reshape(-1, S)
    p = rec[:, 0:12].copy().view(np.float32)
    packed = rec[:, 12:16].copy().view(np.uint32)[:, 0]
    e = np.stack([(packed >> (8 * a)) & 0xFF for a in range(3)], 1).astype(np.uint32)
    scale = (e << 23).view(np.float32)
    imask = packed >> 24
    base = rec[:, 16:24].copy().view(np.uint32)
    hb = rec[:, HB:HB + 4 * width].copy().view(np.uint32)
    q = rec[:, Q:Q + 6 * width].reshape(-1, 6, width).astype(np.float32)
    lo = (q[:, 0:3] * scale[:, :, None]).astype(np.float32) + p[:, :, None]   # q*2^e is exact
    hi = (q[:, 3:6] * scale[:, :, None]).astype(np.float32) + p[:, :, None]
    return dict(p=p, imask=imask, child_base=base[:, 0], tri_base=base[:, 1], hb=hb, lo=lo, hi=hi,
                scale=scale)


def check_tree(v, t, width):
    sc = fgl.Scene(v, t, width=width, upload=False)
    st = sc.stats()
    nodes, tris = sc.export()
    D = decode_nodes(nodes, width)
    ids = tris[:, 3].copy().view(np.int32)
    assert np.array_equal(np.sort(ids), np.arange(len(t)))         # every triangle exactly once
    tv = tris.reshape(-1, 3, 4)[:, :, :3]
    assert np.array_equal(tv, v[t[ids]])                           # leaf records hold the mesh's vertices
    m = st["margin"]
    # content box per node, children (larger index) before parents
    N = st["n_nodes"]
    clo = np.full((N, 3), np.inf)
    chi = np.full((N, 3), -np.inf)
    for ni in range(N - 1, -1, -1):
        for j in range(width):
            hb = int(D["hb"][ni, j])
            if hb == 0:
                continue
            if hb >> 24:
                assert hb == 1 << (24 + j)                             # internal child: bit 24 + slot
                assert (D["imask"][ni] >> j) & 1
                child = int(D["child_base"][ni]) + bin(int(D["imask"][ni]) & ((1 << j) - 1)).count("1")
                assert ni < child < N
                lo, hi = clo[child], chi[child]
            else:
                assert not (D["imask"][ni] >> j) & 1
                off = (hb & -hb).bit_length() - 1
                cnt = bin(hb).count("1")
                assert 1 <= cnt <= 3 and hb >> off == (1 << cnt) - 1   # a short contiguous run
                k = int(D["tri_base"][ni]) + off
                pts = tv[k:k + cnt].reshape(-1, 3).astype(np.float64)
                lo, hi = pts.min(0), pts.max(0)
            g = m + D["scale"][ni].astype(np.float64)        # margin + one quantum
            assert np.all(D["lo"][ni, :, j].astype(np.float64) <= lo - g), (ni, j)
            assert np.all(D["hi"][ni, :, j].astype(np.float64) >= hi + g), (ni, j)
            clo[ni] = np.minimum(clo[ni], lo)
            chi[ni] = np.maximum(chi[ni], hi)
    assert sc.verify() == 0
    return st


@pytest.mark.parametrize("width", [8, 4])
def test_builder_boxes_conservative_tiny_room(width):
    v, t, _ = synth.tiny_room_scene(1)
    st = check_tree(v, t, width)
    assert st["width"] == width and st["node_stride"] == (112 if width == 8 else 64)


@pytest.mark.parametrize("width", [8, 4])
def test_builder_boxes_conservative_random_soup(width):
    rng = np.random.default_rng(3)
    c = rng.uniform(-30, 30, (3000, 1, 3))
    v = (c + rng.uniform(0.001, 2.0, (3000, 1, 1)) * rng.standard_normal((3000, 3, 3))).reshape(-1, 3)
    v = v.astype(np.float32)
    t = np.arange(len(v), dtype=np.int32).reshape(-1, 3)
    check_tree(v, t, width)


def test_builder_degenerate_inputs():
    # single triangle, zero-area triangles, duplicates, many coincident triangles
    v1 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    check_tree(v1, np.array([[0, 1, 2]], np.int32), 8)
    vd = np.zeros((3, 3), np.float32)
    check_tree(vd, np.zeros((5, 3), np.int32), 8)
    check_tree(v1, np.tile(np.array([[0, 1, 2]], np.int32), (5000, 1)), 8)
    check_tree(v1, np.tile(np.array([[0, 1, 2]], np.int32), (5000, 1)), 4)
    # huge and tiny coordinates together
    vb = np.array([[1e4, 1e4, 1e4], [1e4 + 1e-3, 1e4, 1e4], [1e4, 1e4 + 1e-3, 1e4],
                   [-1e4, 0, 0], [-1e4, 1, 0], [-1e4, 0, 1]], np.float32)
    check_tree(vb, np.array([[0, 1, 2], [3, 4, 5]], np.int32), 8)


def test_builder_sah_no_worse_than_median():
    v, t, _ = synth.tiny_room_scene(2)
    sc = fgl.Scene(v, t, upload=False)
    st = sc.stats()
    assert st["depth"] <= 6 and st["sah_cost"] > 0


def test_builder_rejects_bad_input():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    with pytest.raises(fgl.FglError) as e:
        fgl.Scene(v, np.array([[0, 1, 3]], np.int32), upload=False)
    assert e.value.status == fgl.FGL_ERR_INVALID
    vn = v.copy()
    vn[1, 2] = np.nan
    with pytest.raises(fgl.FglError):
        fgl.Scene(vn, np.array([[0, 1, 2]], np.int32), upload=False)
    with pytest.raises(fgl.FglError):
        fgl.Scene(v, np.zeros((0, 3), np.int32), upload=False)
    with pytest.raises(fgl.FglError):
        fgl.Scene(v, np.array([[0, 1, 2]], np.int32), width=5, upload=False)


def test_cast_argument_validation_without_gpu():
    L = fgl.lib()
    v, t, _ = synth.tiny_room_scene(1)
    sc = fgl.Scene(v, t, upload=False)
    P = ctypes.c_void_p
    # null sensor / non-resident scene are rejected before any CUDA call
    st = L.fgl_cast(sc.handle, None, None, 1, 10.0, None, None, None)
    assert st == fgl.FGL_ERR_INVALID
    assert b"null" in L.fgl_last_error()
    item = fgl.CastItem(sc.handle, None, None, 1, 10.0, None, None)
    assert L.fgl_cast_batched(ctypes.byref(item), 1, None, None) == fgl.FGL_ERR_INVALID
    assert L.fgl_cast_batched(None, -1, None, None) == fgl.FGL_ERR_INVALID
    out = P()
    assert L.fgl_sensor_create(None, None, 0, 1, 0, 0, 0, ctypes.byref(out)) == fgl.FGL_ERR_INVALID
    el = np.zeros(6, np.float32)
    assert L.fgl_sensor_create(el.ctypes.data, el.ctypes.data, 6, 4, 2, 0, 0,
                               ctypes.byref(out)) == fgl.FGL_ERR_INVALID   # rows*cols != n
    el[2] = np.inf
    assert L.fgl_sensor_create(el.ctypes.data, el.ctypes.data, 6, 1, 6, 0, 0,
                               ctypes.byref(out)) == fgl.FGL_ERR_INVALID


def test_mesh_argument_validation_without_gpu():
    """fgl_denoise / fgl_tsdf / fgl_marching_tets reject bad arguments before
    any CUDA call."""
    L = fgl.lib()
    F, I = ctypes.c_float, ctypes.c_int32
    good = fgl.Grid((F * 3)(0, 0, 0), 0.1, (I * 3)(4, 4, 4), 0)
    bad_dims = fgl.Grid((F * 3)(0, 0, 0), 0.1, (I * 3)(4, 0, 4), 0)
    bad_h = fgl.Grid((F * 3)(0, 0, 0), float("nan"), (I * 3)(4, 4, 4), 0)
    huge = fgl.Grid((F * 3)(0, 0, 0), 0.1, (I * 3)(2048, 2048, 1024), 0)
    fake = ctypes.c_void_p(16)                      # never dereferenced: rejected first
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    E = fgl.FGL_ERR_INVALID
    assert L.fgl_tsdf(None, ctypes.byref(good), 0.1, fake, None, None, None, None) == E
    assert L.fgl_tsdf(fake, ctypes.byref(bad_dims), 0.1, fake, None, None, None, None) == E
    assert L.fgl_tsdf(fake, ctypes.byref(bad_h), 0.1, fake, None, None, None, None) == E
    assert L.fgl_tsdf(fake, ctypes.byref(good), 0.0, fake, None, None, None, None) == E
    assert L.fgl_tsdf(fake, ctypes.byref(good), 26.0, fake, None, None, None, None) == E   # 260 shells
    assert L.fgl_tsdf(fake, ctypes.byref(huge), 0.1, fake, None, None, None, None) == E
    assert L.fgl_denoise(fake, ctypes.byref(good), 0.0, 0, 0.5, None, fake, None, None) == E
    assert L.fgl_denoise(fake, ctypes.byref(good), 0.1, 2, 0.5, None, fake, None, None) == E
    assert L.fgl_denoise(fake, ctypes.byref(good), 0.1, 1, 1.5, None, fake, None, None) == E
    assert L.fgl_denoise(fake, ctypes.byref(good), 5.0, 0, 0.5, None, fake, None, None) == E  # 150 taps
    assert L.fgl_denoise(fake, ctypes.byref(good), 0.1, 0, 0.5, None, None, None, None) == E
    assert L.fgl_marching_tets(fake, ctypes.byref(good), 0.0, 0, None, 0, None, 0, None,
                               ctypes.byref(nv), ctypes.byref(nt), None) == E
    assert L.fgl_marching_tets(fake, ctypes.byref(good), float("inf"), 1, None, 0, None, 0, None,
                               ctypes.byref(nv), ctypes.byref(nt), None) == E
    assert L.fgl_marching_tets(fake, ctypes.byref(good), 0.0, 1, fake, 4, None, 4, None,
                               ctypes.byref(nv), ctypes.byref(nt), None) == E
    assert L.fgl_marching_tets(None, ctypes.byref(good), 0.0, 1, None, 0, None, 0, None,
                               ctypes.byref(nv), ctypes.byref(nt), None) == E


def test_checked_library_loads_and_exports_every_declared_symbol():
    """FGL_CHECKED=1 makes the binding load the bounds-checked build
    (libfgl_checked.so), which exports the same C ABI.  A child process, since
    a process loads one of the two libraries."""
    import subprocess
    import sys
    from paper_2509_17390_gb300 import build_native
    build_native.build(checked=True)
    code = ("import json, paper_2509_17390_gb300 as f; L = f.lib(); "
            "import sys; names = json.loads(sys.argv[1]); "
            "missing = [n for n in names if not hasattr(L, n)]; "
            "print(L._name); assert not missing, missing")
    import json
    r = subprocess.run([sys.executable, "-c", code, json.dumps(declared_functions())], cwd=ROOT,
                       env=dict(os.environ, FGL_CHECKED="1"), capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().endswith("libfgl_checked.so")
