"""The cast workloads test_gpu_checked.py runs through both the production
library and the checked one (libfgl_checked.so's bounds-checked traversal):
every kernel family that reads scene nodes and triangles -- plain and
batched, widths 8 and 4, pooled and lane-serial leaf tests, a two-entry
shared-memory stack that sends most pushes down the spill path, t_min, the
fused and the per-instance instance passes, the LBVH.  Called with the
package and torch of the process (one process loads one library)."""

import numpy as np

import synth
from synth import workloads


def _rot_z(a):
    return np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])


def run_cases(fgl, torch) -> dict:
    out = {}
    cu = lambda a, dt=np.float32: torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()

    def keep(name, r, i):
        fgl.sync()
        out[name + "_range"] = r.cpu().numpy()
        out[name + "_tri"] = i.cpu().numpy()

    w = workloads.indoor_scan(2)
    rng = np.random.default_rng(3)
    P = cu(synth.sample_free_pose(rng, w.obstacles, 24, upright=False))
    se = fgl.Sensor.from_table(synth.grid_sensor(16, -15, 15, 360))
    n = 24 * se.n_rays
    for width in (8, 4):
        sc = fgl.Scene(w.verts, w.tris, width=width)
        keep(f"plain{width}", *fgl.cast(sc, se, P, 120.0))
        for tri_mode, sdepth in ((0, 0), (1, 0), (0, 2), (1, 2)):
            r = torch.empty(n, device="cuda")
            i = torch.empty(n, dtype=torch.int32, device="cuda")
            fgl.cast_batched([(sc, se, P, 120.0, r, i, 0.4)],
                             fgl.BatchOpts(tri_mode=tri_mode, stack_smem=sdepth))
            keep(f"batched{width}_{tri_mode}_{sdepth}", r, i)

    # instances: one width (fused launch) and mixed widths (one pass each)
    vs, ts, obs = synth.tiny_room_scene(9)
    uv, ut = synth.icosphere_unit(2)
    meshes = [((0.35 * uv).astype(np.float32), ut),
              synth.aabb_box((-0.3, -0.2, -0.25), (0.3, 0.2, 0.25), 2),
              synth.aabb_box((-0.1, -0.1, -0.6), (0.1, 0.1, 0.6), 1)]
    Pi = synth.sample_free_pose(rng, obs, 8)
    IP = np.zeros((8, 3, 3, 4), np.float32)
    for e in range(8):
        for k in range(3):
            IP[e, k, :, :3] = _rot_z(rng.uniform(0, 2 * np.pi))
            IP[e, k, :, 3] = Pi[e, :, 3] + rng.uniform(-2.5, 2.5, 3) * [1, 1, 0.3] + [0, 0, 0.1]
    scene = fgl.Scene(vs, ts)
    ni = 8 * se.n_rays
    for name, widths in (("fused", (8, 8, 8)), ("mixed", (8, 4, 8))):
        inst = [fgl.Scene(v, t, width=wd) for (v, t), wd in zip(meshes, widths)]
        r = torch.empty(ni, device="cuda")
        i = torch.empty(ni, dtype=torch.int32, device="cuda")
        k = torch.empty(ni, dtype=torch.int32, device="cuda")
        fgl.cast_batched([(scene, se, cu(Pi), 100.0, r, i, 0.0,
                           {"instances": inst, "instance_poses": cu(IP), "out_instance": k})])
        keep("inst_" + name, r, i)
        out["inst_" + name + "_k"] = k.cpu().numpy()

    # the GPU-built LBVH
    lb = fgl.Lbvh(cu(w.verts), cu(w.tris, np.int32))
    keep("lbvh", *lb.cast(se, P, 120.0, min_range=0.4))
    out["lbvh_overflow"] = np.array([lb.stats()["overflow"]])
    return out
