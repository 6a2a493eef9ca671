"""Independent FP64 restatement of the slice geometry for the oracle pins.

Written from the paper's statement of the method (Algorithm 1, Section 3.1)
for tiny inputs only, so that the C oracle can be checked against something
other than itself.  Sampling here assumes zero noise (xi_phi = xi_s = 0).
"""
import math

import numpy as np


def f32(x):
    return np.float32(x)


def sample_offsets(radius, fx, z, ns, step_mode=0):
    """Offsets (pixels) of the N_s steps, in binary32 as the sample pixel is chosen (xi_s = 0)."""
    rpx = f32(min(f32(f32(radius) * f32(fx)) / f32(z), f32(1048576.0)))
    dn = f32(f32(1.0) / f32(ns + 1))
    out = []
    for j in range(ns):
        if step_mode == 0:
            out.append(f32(f32(j + 1) * f32(rpx * dn)))
        else:
            uj = f32(f32(j + 1) * dn)
            out.append(f32(f32(uj * uj) * rpx))
    return out


def slice_dir(i, nd):
    phi = i * math.pi / nd
    return f32(math.cos(phi)), f32(math.sin(phi))


def unproject(cam, u, v, z):
    return np.array([(u - cam.cx) / cam.fx * z, -(v - cam.cy) / cam.fy * z, -z], dtype=np.float64)


def frame(cam, x, y, z, n, cphi, sphi):
    """p, v (unit, toward the camera), s (unit, in-slice toward +omega), gamma."""
    p = unproject(cam, x + 0.5, y + 0.5, float(z))
    v = -p / np.linalg.norm(p)
    w3 = np.array([float(cphi) / cam.fx, -float(sphi) / cam.fy, 0.0])
    s = w3 - np.dot(w3, v) * v
    s /= np.linalg.norm(s)
    nv, ns_ = float(np.dot(n, v)), float(np.dot(n, s))
    gamma = math.atan2(ns_, nv) if (nv != 0 or ns_ != 0) else 0.0
    return p, v, s, gamma


def sector_coord(h, gamma, nb):
    return min(max((h - gamma) * nb / math.pi + nb / 2.0, 0.0), float(nb))


def half_covered_mask(A, B, nb):
    m = 0
    for k in range(nb):
        if min(B, k + 1) - max(A, k) >= 0.5:
            m |= 1 << k
    return m


def sample_pixels(x, y, W, H, depth, offs, cphi, sphi, sigma):
    """(qx, qy) of the steps that read geometry, near to far, for one side."""
    out = []
    for o in offs:
        # nearest integer (ties to even) of the exact binary32 product
        dx = float(np.rint(float(o) * float(f32(sigma * cphi))))
        dy = float(np.rint(float(o) * float(f32(sigma * sphi))))
        if dx == 0 and dy == 0:
            continue
        qx, qy = x + int(dx), y + int(dy)
        if not (0 <= qx < W and 0 <= qy < H):
            continue
        zq = float(depth[qy, qx])
        if not (0 < zq < math.inf):
            continue
        out.append((qx, qy, zq))
    return out
