"""CPU-side checks of the C-ABI library: it loads, exports every entry point
include/fgl.h declares, validates arguments, and its host BVH builder makes
conservative child boxes (checked here independently of the library's
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
    """Node records as laid out by the builder: a 32-byte header (corner p,
    imask, child_base, tri_base), six blocks of `width` float offsets (lo x,
    y, z, hi x, y, z), then the hit bits: 256 B for width 8, 144 B for 4."""
    S = 32 + 28 * width
    rec = nodes.reshape(-1, S)
    p = rec[:, 0:12].copy().view(np.float32)
    imask = rec[:, 12:16].copy().view(np.uint32)[:, 0]
    base = rec[:, 16:24].copy().view(np.uint32)
    off = rec[:, 32:32 + 24 * width].copy().view(np.float32).reshape(-1, 6, width).astype(np.float64)
    hb = rec[:, 32 + 24 * width:S].copy().view(np.uint32)
    lo = p[:, :, None].astype(np.float64) + off[:, 0:3]     # summed in double, as the builder checks
    hi = p[:, :, None].astype(np.float64) + off[:, 3:6]
    return dict(p=p, imask=imask, child_base=base[:, 0], tri_base=base[:, 1], hb=hb, lo=lo, hi=hi)


def check_tree(v, t, width, want_boxes=False):
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
    boxes = []
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
            assert np.all(D["lo"][ni, :, j] <= lo - m), (ni, j)       # content grown by the margin
            assert np.all(D["hi"][ni, :, j] >= hi + m), (ni, j)
            clo[ni] = np.minimum(clo[ni], lo)
            chi[ni] = np.maximum(chi[ni], hi)
            boxes.append((ni, j, lo, hi))
    assert sc.verify() == 0
    return (st, D, boxes) if want_boxes else st


@pytest.mark.parametrize("width", [8, 4])
def test_builder_boxes_conservative_tiny_room(width):
    v, t, _ = synth.tiny_room_scene(1)
    st = check_tree(v, t, width)
    assert st["width"] == width and st["node_stride"] == (256 if width == 8 else 144)


@pytest.mark.parametrize("width", [8, 4])
def test_builder_boxes_conservative_random_soup(width):
    rng = np.random.default_rng(3)
    c = rng.uniform(-30, 30, (3000, 1, 3))
    v = (c + rng.uniform(0.001, 2.0, (3000, 1, 1)) * rng.standard_normal((3000, 3, 3))).reshape(-1, 3)
    v = v.astype(np.float32)
    t = np.arange(len(v), dtype=np.int32).reshape(-1, 3)
    check_tree(v, t, width)


def _f32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def _slab_hits_f32(D, ni, j, o, ix, tmax):
    """The traversal's slab test of child slot j of node ni in float32:
    t = fma(off, 1/d, (p - o) * (1/d)) per plane (the product of two floats is
    exact in double, then one rounding), near plane by the sign of 1/d."""
    p = D["p"][ni].astype(np.float64)
    lo = D["lo"][ni, :, j] - p          # the stored offsets
    hi = D["hi"][ni, :, j] - p
    B = _f32(_f32(p[None] - o) * ix)
    tlo = _f32(lo[None] * ix + B)
    thi = _f32(hi[None] * ix + B)
    near = np.where(ix < 0, thi, tlo)
    far = np.where(ix < 0, tlo, thi)
    tn = np.maximum(near.max(1), 0.0)
    tf = np.minimum(far.min(1), tmax)
    return tn <= tf


def _rays_at_box(rng, lo, hi, slo, shi, k):
    """k rays from origins anywhere in the scene box [slo, shi] aimed at points
    on the surface of [lo, hi] (faces, edges and corners): float32 origin and
    direction, approximate reciprocal within 2^-22 as on the device."""
    tgt = rng.uniform(lo, hi, (k, 3))
    ax = rng.integers(0, 3, k)
    side = rng.integers(0, 2, k)
    tgt[np.arange(k), ax] = np.where(side == 1, hi[ax], lo[ax])
    corner = rng.random(k) < 0.25
    tgt[corner] = np.where(rng.integers(0, 2, (int(corner.sum()), 3)) == 1, hi, lo)
    o = _f32(rng.uniform(slo, shi, (k, 3)))
    d = _f32(tgt - o)
    d = np.where(np.abs(d) < 1e-20, 1e-20, d)
    ix = _f32(1.0 / d * (1.0 + rng.uniform(-1, 1, (k, 3)) * 2.0 ** -22))
    return o, d, ix


def _true_hits(lo, hi, o, d, tmax):
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo[None] - o) / d
        t2 = (hi[None] - o) / d
    tn = np.maximum(np.minimum(t1, t2).max(1), 0.0)
    tf = np.minimum(np.maximum(t1, t2).min(1), tmax)
    return tn <= tf


@pytest.mark.parametrize("case", ["room", "soup", "far"])
def test_slab_test_conservative_in_float32(case):
    """The stored child boxes with the builder's margin survive the
    traversal's float32 plane arithmetic: every ray that truly meets a
    child's content box (here aimed at its faces, edges and corners, the
    grazing cases) passes the emulated slab test of that child."""
    rng = np.random.default_rng(11)
    if case == "room":
        v, t, _ = synth.tiny_room_scene(1)
    elif case == "soup":
        c = rng.uniform(-30, 30, (1500, 1, 3))
        v = (c + rng.uniform(0.001, 2.0, (1500, 1, 1)) * rng.standard_normal((1500, 3, 3))).reshape(-1, 3)
        t = np.arange(len(v), dtype=np.int32).reshape(-1, 3)
    else:  # small triangles far from the origin
        c = 1e4 + rng.uniform(-5, 5, (600, 1, 3))
        v = (c + 1e-2 * rng.standard_normal((600, 3, 3))).reshape(-1, 3)
        t = np.arange(len(v), dtype=np.int32).reshape(-1, 3)
    v = v.astype(np.float32)
    st, D, boxes = check_tree(v, t, 8, want_boxes=True)
    slo, shi = np.array(st["bounds_lo"], np.float64), np.array(st["bounds_hi"], np.float64)
    tmax = 4.0 * float(np.linalg.norm(shi - slo)) + 1.0
    n_true = 0
    for ni, j, lo, hi in boxes[:4000]:
        o, d, ix = _rays_at_box(rng, lo, hi, slo, shi, 24)
        truth = _true_hits(lo, hi, o, d, tmax)
        got = _slab_hits_f32(D, ni, j, o, ix, tmax)
        n_true += int(truth.sum())
        assert not np.any(truth & ~got), (case, ni, j)
    assert n_true > 1000


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
