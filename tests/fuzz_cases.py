"""Seeded random gather problems for the GPU parity fuzz test: sizes, every parameter the ABI
takes, storage format, noise, SH environment, and camera intrinsics and view rotation perturbed
away from the scene generator's symmetric camera.  Inputs only; both sides read them."""
import dataclasses
import math

import numpy as np

import scenegen
from scenegen import Params


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]], dtype=np.float32)


def case(k: int):
    """Case k: (gbuffer, params, noise for the ABI, noise table for the oracle, sh)."""
    rng = np.random.default_rng(9000 + k)
    W = int(rng.choice([1, 2, 7, 33, 64, 97, 160, 231]))
    H = int(rng.choice([1, 3, 16, 45, 90, 128, 177]))
    g = scenegen.render(9000 + k, W, H, int(rng.integers(4, 24)), int(rng.integers(0, 6)))
    if rng.random() < 0.4:
        g = g.as_f16()
    cam = g.camera
    cam = dataclasses.replace(cam, fx=float(np.float32(cam.fx * rng.uniform(0.4, 2.5))),
                              fy=float(np.float32(cam.fy * rng.uniform(0.4, 2.5))),
                              cx=float(np.float32(cam.cx + rng.uniform(-0.3, 0.3) * W)),
                              cy=float(np.float32(cam.cy + rng.uniform(-0.3, 0.3) * H)),
                              view_to_world=_rotation(rng))
    g = dataclasses.replace(g, camera=cam)
    nb = int(rng.choice([32, 64, 128]))
    cones = int(rng.choice([0, 0, 1, 2, 4, 8]))
    prm = Params(num_slices=int(rng.integers(1, 17)), steps_per_side=int(rng.integers(1, 65)),
                 radius=float(np.float32(rng.uniform(0.05, 6.0))),
                 thickness=math.inf if rng.random() < 0.2 else float(np.float32(rng.uniform(0.01, 3.0))),
                 thickness_slope=float(np.float32(rng.uniform(0.0, 0.1))) if rng.random() < 0.3 else 0.0,
                 sector_count=nb, hit_rule=int(rng.random() < 0.3), ambient_cones=cones,
                 step_mode=int(rng.random() < 0.4), gi=bool(rng.random() < 0.85))
    u = rng.random()
    if u < 0.2:
        noise, table = None, None
    elif u < 0.5:
        frame = int(rng.integers(0, 200))
        noise, table = ("ign", frame), scenegen.ign_table(frame)
    else:
        table = np.minimum(rng.random((16, 2)), 0.99999994).astype(np.float32)
        noise = table
    sh = None
    if cones:
        sh = (rng.uniform(-0.3, 0.3, (9, 3)) + np.array([[0.8, 0.7, 0.6]] + [[0, 0, 0]] * 8)).astype(np.float32)
    return g, prm, noise, table, sh
