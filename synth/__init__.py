"""Seeded synthetic inputs for batched LiDAR ray casting.

This package produces the *inputs* of the ray-casting path (triangle meshes,
sensor beam tables, sensor poses) and nothing else: it holds none of the
ray-casting arithmetic.  Both the CUDA library and the CPU oracle consume what
it makes, which is why it is a package of its own.

Everything is drawn from ``numpy.random.default_rng(seed)``; the same seed in
the same process gives the same arrays.

Conventions (shared by every consumer):
  * vertices: float32 [nv, 3] in metres; triangles: int32 [nt, 3] vertex ids.
  * sensor beam table: float32 elevation and azimuth in radians, one entry per
    ray, row-major over (beam row, azimuth column) for grid sensors.
  * poses: float32 [n_env, 3, 4] row-major ``[R | t]`` (sensor -> world), the
    pose T_s of the LiDAR measurement model (paper Sec. IV-C, eq. r_j).
"""

from .scenes import (  # noqa: F401
    box_room,
    aabb_box,
    icosphere_unit,
    merge_meshes,
    tiny_room_scene,
    indoor_scene,
    Obstacles,
)
from .sensors import grid_sensor, rosette_sensor, SensorTable  # noqa: F401
from .poses import (  # noqa: F401
    pose_from_yaw,
    random_rotation,
    sample_free_pose,
    random_walk,
)
