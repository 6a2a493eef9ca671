"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each expected value comes from
a closed form, a hand-worked fixture, a brute-force restatement on a tiny
input, or an invariant the method must satisfy (Section 3.1-3.3).
"""
import math
import os

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import Params
from tests import _geom as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = float("inf")


def _read_cases():
    rows = []
    with open(os.path.join(GOLDEN, "sector_rule_cases.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                nb, rule, A, B, m = line.split()
                rows.append((int(nb), int(rule), float(A), float(B), int(m, 16)))
    return rows


# --- hit rule (Section 3.1 round criterion, Figure 4, Algorithm 1) -------------------------

@pytest.mark.parametrize("nb,rule,A,B,expect", _read_cases())
def test_hit_rule_hand_cases(nb, rule, A, B, expect):
    assert oracle.sector_mask_words(A, B, nb, rule, fp64=True) == expect
    assert oracle.sector_mask_words(A, B, nb, rule) == expect


@pytest.mark.parametrize("nb", [32, 64, 128])
@pytest.mark.parametrize("rule", [0, 1])
def test_hit_rule_o1_equals_per_sector(nb, rule):
    """The O(1) run of ones equals the per-sector brute force on a grid of exact endpoints,
    including every tie (endpoints on sector centres and widths of exactly 1/2)."""
    step = {32: 1.0 / 8.0, 64: 1.0 / 4.0, 128: 1.0 / 2.0}[nb]
    vals = np.arange(0.0, nb + step / 2, step)
    fine = np.arange(0.0, 2.5, 1.0 / 128.0)
    for grid in (vals, fine):
        for A in grid:
            for B in grid[grid >= A]:
                a, b = float(A), float(B)
                assert oracle.sector_mask_words(a, b, nb, rule) == oracle.sector_mask_words(a, b, nb, rule, True), (a, b)


def test_hit_rule_random_endpoints():
    rng = np.random.default_rng(5)
    for _ in range(20000):
        A, B = np.sort(rng.uniform(0, 32, 2).astype(np.float32))
        m32 = oracle.sector_mask32(float(A), float(B), 32, 0)
        assert m32 == G.half_covered_mask(float(A), float(B), 32)


# --- own arithmetic of the binary32 replica ---------------------------------------------------

def test_acos_error_bound_exhaustive():
    """Every binary32 in [0, 1]: within 3e-7 rad of the libm double acos (A&S 4.4.46 bounds
    the exact-arithmetic error by 2e-8; the rest is binary32 rounding).  The sweep also
    counts increases: the binary32 evaluation is not strictly monotone (one-ulp upticks)."""
    err, inc = oracle.acos32_sweep(64)
    assert err < 3e-7
    assert inc < 5000
    for x in (-1.0, -0.5, 0.0, 0.5, 1.0):
        assert abs(oracle.acos32(x) - math.acos(x)) < 3e-7
    assert oracle.acos32(1.0) == 0.0


def test_rsqrt_error_bound():
    assert oracle.rsqrt32_sweep(1e-37, 1e37, 200000) < 3e-7
    assert oracle.rsqrt32_sweep(0.5, 8.0, 200000) < 3e-7
    assert math.isfinite(oracle.rsqrt32(0.0))


# --- flat plane and empty sky (Section 3.1: samples in the tangent plane occlude nothing) ------

@pytest.mark.parametrize("normal", [(0.0, 0.0, 1.0), (0.0, 0.6, 0.8), (0.5, -0.3, 0.81), (-0.9, 0.1, 0.42)])
@pytest.mark.parametrize("thickness", [0.5, INF])
def test_flat_plane_no_occlusion(normal, thickness):
    """Slices at multiples of pi/4 sample pixels on the slice line, so every sample lies in the
    plane of the centre pixel: no sector is half covered, AO = 1 and GI = 0 exactly."""
    g = scenegen.hand_plane(41, 33, normal_view=normal, point_depth=6.0)
    prm = Params(num_slices=4, steps_per_side=7, radius=2.0, thickness=thickness)
    for fn in (oracle.fp64, oracle.fp32):
        res = fn(oracle.Problem(g, prm, None))
        o0, masks = res[0], res[2]
        geo = np.isfinite(g.depth.ravel())
        assert geo.sum() > 100
        assert np.all(masks == 0)
        assert np.all(o0[:, 3] == 1.0)
        assert np.all(o0[:, :3] == 0.0)


def test_quad_over_sky_full_visibility():
    g = scenegen.hand_quad_over_sky(48, 40)
    prm = Params(num_slices=4, steps_per_side=8, radius=1.5, thickness=0.3, ambient_cones=0)
    for fn in (oracle.fp64, oracle.fp32):
        o0, o1, masks = fn(oracle.Problem(g, prm, None))[:3]
        assert np.all(masks == 0) and np.all(o0[:, 3] == 1.0) and np.all(o0[:, :3] == 0.0)


def test_sky_pixels_fully_visible():
    g = scenegen.hand_quad_over_sky(20, 20, x0=5, x1=10, y0=5, y1=10)
    prm = Params(num_slices=3, steps_per_side=4)
    o0, o1, masks, _ = oracle.fp64(oracle.Problem(g, prm, scenegen.ign_table()))
    sky = ~np.isfinite(g.depth.ravel())
    assert np.all(o0[sky] == [0, 0, 0, 1]) and np.all(o1[sky] == 0) and np.all(masks[sky] == 0)


# --- infinite thickness is the horizon method quantised to sectors (Section 3.1) -------------

def _horizon_masks(g, nd, ns, radius, nb):
    """GTAO-style horizons (largest cosine per side over the same samples), quantised by the
    half-covered rule; restated here in FP64 from the definition."""
    H, W = g.depth.shape
    cam = g.camera
    out = np.zeros((H * W, nd), dtype=object if nb == 128 else np.uint64)
    for y in range(H):
        for x in range(W):
            z = float(g.depth[y, x])
            if not (0 < z < INF):
                continue
            n = g.normal[y, x, :3].astype(np.float64)
            offs = G.sample_offsets(radius, cam.fx, z, ns)
            for i in range(nd):
                cphi, sphi = G.slice_dir(i, nd)
                p, v, s, gamma = G.frame(cam, x, y, z, n, cphi, sphi)
                m = 0
                for sigma in (-1, 1):
                    best = -INF
                    for qx, qy, zq in G.sample_pixels(x, y, W, H, g.depth, offs, cphi, sphi, sigma):
                        l = G.unproject(cam, qx + 0.5, qy + 0.5, zq) - p
                        best = max(best, float(np.dot(l, v) / np.linalg.norm(l)))
                    if best == -INF:
                        continue
                    h = sigma * math.acos(max(-1.0, min(1.0, best)))
                    X = G.sector_coord(h, gamma, nb)
                    m |= G.half_covered_mask(X, nb, nb) if sigma > 0 else G.half_covered_mask(0.0, X, nb)
                out[y * W + x, i] = m
    return out


@pytest.mark.parametrize("nb", [32, 64, 128])
def test_infinite_thickness_equals_quantised_horizon(nb):
    g = scenegen.render(11, 28, 22, 6, 2)
    prm = Params(num_slices=2, steps_per_side=6, radius=3.0, thickness=INF, sector_count=nb)
    _, _, masks, margin = oracle.fp64(oracle.Problem(g, prm, None))
    ref = _horizon_masks(g, 2, 6, 3.0, nb)
    assert np.count_nonzero(ref) > 20
    if nb == 128:
        masks = masks[..., 0].astype(object) | (masks[..., 1].astype(object) << 64)
        ref = ref.astype(object)
    diff = masks != ref
    assert np.all(margin[diff] < 1e-9)
    assert diff.mean() < 1e-3


# --- single infinite wall: closed-form occluded fraction (Section 3.1) ------------------------

@pytest.mark.parametrize("axis,xi", [(0, None), (1, None), (0, (0.37, 0.5)), (1, (0.37, 0.25))])
@pytest.mark.parametrize("thickness", [INF, 2.0])
def test_step_wall_closed_form(thickness, axis, xi):
    """Centre pixel on the back plane at the principal point (gamma = 0).  A wall face at
    x = X_w (axis 0), or a ledge edge at y = -X_w below the centre (axis 1), rises H_w toward
    the camera.  Slice phi steps along (cos phi, sin phi) in pixels with image y down, i.e.
    along view (cos phi, -sin phi); with c the component of that direction toward the step,
    its top edge is at in-plane distance X_w/|c|, and the occluded sectors are the
    N_b (pi/2 - h*)/pi nearest the hemisphere edge of the side facing it (sectors N_b-1 down
    for side +omega, 0 up for side -omega), h* = atan2(X_w/|c|, H_w).  Holds for t = inf and
    any t >= H_w, as long as the samples reach the top edge.  With a noise table, slice i lies at
    (i + xi_phi) pi / N_d and the steps are jittered by xi_s (Algorithm 1, directions and steps
    with random offsets): no slice is then parallel to the step, and every one must see it at its
    rotated angle."""
    W = H = 255
    z0, xw, hw, nb = 4.0, 0.6, 1.5, 32
    g = scenegen.hand_step_wall(W, H, z0, xw, hw, axis=axis)
    radius = 3.0 if xi is None else 4.0  # oblique slices need the longer reach
    prm = Params(num_slices=4, steps_per_side=48, radius=radius, thickness=thickness, sector_count=nb)
    c = (W - 1) // 2
    noise = None
    if xi is not None:
        noise = np.zeros((16, 2), dtype=np.float32)
        noise[(c & 3) * 4 + (c & 3)] = xi  # the centre pixel's class
    _, _, masks, _ = oracle.fp64(oracle.Problem(g, prm, noise), pixels=[(c, c)])
    half = (1 << (nb // 2)) - 1
    for i in range(4):
        phi = (i + (0.0 if xi is None else float(np.float32(xi[0])))) * math.pi / 4
        toward = math.cos(phi) if axis == 0 else math.sin(phi)  # +x, or -y in view space
        m = int(masks[0, i])
        if abs(toward) < 1e-9:
            assert m == 0, (i, hex(m))
            continue
        # the last step reaches past the top edge: its pixel offset toward the step exceeds the
        # edge's, xw / (z0 - hw) * f / |c| pixels along the slice
        assert radius * g.camera.fx / z0 * 48 / 49 > xw / (z0 - hw) * g.camera.fx / abs(toward)
        expect = nb * (math.pi / 2 - math.atan2(xw / abs(toward), hw)) / math.pi
        assert abs(bin(m).count("1") - expect) <= 1.0, (i, bin(m).count("1"), expect)
        if toward > 0:   # side +omega faces the step: a run ending at sector N_b - 1
            assert m & half == 0 and m >> (nb - 1) == 1, (i, hex(m))
        else:            # side -omega faces it: a run starting at sector 0
            assert m >> (nb // 2) == 0 and m & 1 == 1, (i, hex(m))


# --- single sample: closed-form indirect light (Algorithm 1 GI line, Section 3.3) -------------

@pytest.mark.parametrize("step_mode,step,nb,slope,nd", [(0, 0, 32, 0.0, 1), (1, 2, 32, 0.0, 1), (0, 1, 128, 0.05, 1),
                                                       (1, 3, 64, 0.05, 1), (0, 0, 32, 0.0, 2)])
def test_single_sample_gi_closed_form(step_mode, step, nb, slope, nd):
    """Sky everywhere except the centre pixel p and one pixel q on step `step` of the +omega
    side of slice 0 (constant steps, or quadratic steps r ((j+1)/(N_s+1))^2: the reading taken of
    the growing step lengths of Section 4.3).
    The result is that sample alone: cnt sectors of its slab,
    GI = cnt/N_b * c_q * max(0, n_p.l) * max(0, -n_q.l) / N_d.  Also for 64 and 128 sectors
    (sector k is bit k % 64 of word k / 64), a thickness t0 + slope z_p growing with depth, and
    N_d = 2, whose second (vertical) slice sees only sky: GI and occlusion are averaged over the
    slices."""
    W = H = 31
    fx = 15.5
    cam = scenegen.Camera(fx, fx, 15.5, 15.5)
    c = 15
    radius, ns, t0 = 2.0, 4, 0.4
    z, zq = 3.0, 2.2
    t = float(np.float32(t0)) + float(np.float32(slope)) * z
    offs = G.sample_offsets(radius, fx, z, ns, step_mode=step_mode)
    dq = int(np.rint(offs[step]))
    assert dq >= 1 and all(int(np.rint(o)) != dq for k, o in enumerate(offs) if k != step)
    depth = np.full((H, W), np.inf, dtype=np.float32)
    depth[c, c] = z
    depth[c, c + dq] = zq
    nrm = np.zeros((H, W, 4), dtype=np.float32)
    nrm[c, c, :3] = (0.0, 0.0, 1.0)
    nq = np.array([-0.6, 0.0, 0.8], dtype=np.float32)
    nrm[c, c + dq, :3] = nq
    rad = np.zeros((H, W, 4), dtype=np.float32)
    cq = np.array([0.9, 0.4, 0.2], dtype=np.float32)
    rad[c, c + dq, :3] = cq
    g = scenegen.GBuffer(depth, nrm, rad, cam)
    prm = Params(num_slices=nd, steps_per_side=ns, radius=radius, thickness=t0, thickness_slope=slope,
                 sector_count=nb, step_mode=step_mode)

    # closed form
    n_p = np.array([0.0, 0.0, 1.0])
    p, v, s, gamma = G.frame(cam, c, c, z, n_p, np.float32(1.0), np.float32(0.0))
    sf = G.unproject(cam, c + dq + 0.5, c + 0.5, zq)
    l = sf - p
    hf = math.acos(np.dot(l, v) / np.linalg.norm(l))
    sb = sf + t * p / np.linalg.norm(p)
    lb = sb - p
    hb = math.acos(np.dot(lb, v) / np.linalg.norm(lb))
    A, B = sorted([G.sector_coord(hf, gamma, nb), G.sector_coord(hb, gamma, nb)])
    m = G.half_covered_mask(A, B, nb)
    cnt = bin(m).count("1")
    assert cnt >= 2
    lh = l / np.linalg.norm(l)
    w = cnt / nb * max(0.0, float(np.dot(n_p, lh))) * max(0.0, float(-np.dot(nq.astype(np.float64), lh)))
    gi = w * cq.astype(np.float64) / nd
    ao = (1.0 - cnt / nb + (nd - 1)) / nd  # the other slice (vertical) sees only sky

    def as_int(words):
        words = np.atleast_1d(words)
        return sum(int(wd) << (64 * i) for i, wd in enumerate(words))

    o0, _, masks, _, ratio = oracle.fp64(oracle.Problem(g, prm, None), pixels=[(c, c)], ratio=True)
    assert as_int(masks[0, 0]) == m
    assert all(as_int(masks[0, i]) == 0 for i in range(1, nd))
    np.testing.assert_allclose(o0[0, :3], gi, rtol=1e-12, atol=1e-15)
    assert abs(o0[0, 3] - ao) < 1e-15
    # the replica must take the same decisions: each lies beyond its binary32 error bound
    assert ratio[0, 0] > 1.0
    r0, _, rmask = oracle.fp32(oracle.Problem(g, prm, None), pixels=[(c, c)])
    assert as_int(rmask[0, 0]) == m
    np.testing.assert_allclose(r0[0, :3], gi, atol=2e-6)


def test_a_sector_both_sides_cover_is_credited_to_the_minus_side():
    """Under the floor/ceil rule both sides of a slice can set the sector that straddles the split
    between them.  Side -omega runs first, then side +omega (near to far within each side,
    Section 3.3 credits a sector to the first sample that sets it), so that sector's indirect
    light comes from the -omega sample.  One sample on each side, just off the view ray and far in
    front of p, with different radiance; gamma puts the split in the middle of sector N_b/2 - 1.
    The -omega sample is credited ceil(X_f-) sectors, the +omega one N_b - floor(X_f+) - 1;
    crediting +omega first, or both, gives a different GI."""
    W = H = 31
    fx = 15.5
    cam = scenegen.Camera(fx, fx, 15.5, 15.5)
    c, d = 15, 2
    nb = 32
    z, zq = float(np.float32(7.45)), 1.0  # the depths as stored (binary32)
    gam = math.pi / (2 * nb)
    n_p = np.array([math.sin(gam), 0.0, math.cos(gam)], dtype=np.float32)
    radius = float(np.float32(2 * d * z / fx))
    offs = G.sample_offsets(radius, fx, z, 1)
    assert int(np.rint(offs[0])) == d
    depth = np.full((H, W), np.inf, dtype=np.float32)
    depth[c, c] = z
    nrm = np.zeros((H, W, 4), dtype=np.float32)
    nrm[c, c, :3] = n_p
    rad = np.zeros((H, W, 4), dtype=np.float32)
    cols = {-1: np.array([0.9, 0.2, 0.1], dtype=np.float32), 1: np.array([0.1, 0.3, 0.8], dtype=np.float32)}
    nq = np.array([0.0, 0.0, -1.0], dtype=np.float32)
    for sigma in (-1, 1):
        depth[c, c + sigma * d] = zq
        nrm[c, c + sigma * d, :3] = nq
        rad[c, c + sigma * d, :3] = cols[sigma]
    g = scenegen.GBuffer(depth, nrm, rad, cam)
    prm = Params(num_slices=1, steps_per_side=1, radius=radius, thickness=INF, sector_count=nb, hit_rule=1)

    # closed form: t = infinity puts each back endpoint on its side's hemisphere edge
    p, v, s, gamma = G.frame(cam, c, c, z, n_p.astype(np.float64), np.float32(1.0), np.float32(0.0))
    assert abs(gamma - gam) < 1e-7
    X, w = {}, {}
    for sigma in (-1, 1):
        l = G.unproject(cam, c + sigma * d + 0.5, c + 0.5, zq) - p
        lh = l / np.linalg.norm(l)
        X[sigma] = G.sector_coord(sigma * math.acos(float(np.dot(lh, v))), gamma, nb)
        w[sigma] = (max(0.0, float(np.dot(n_p, lh))) * max(0.0, float(-np.dot(nq, lh))) / nb
                    * cols[sigma].astype(np.float64))
    assert nb / 2 - 1 < X[-1] < nb / 2 - 0.5 < X[1] < nb / 2  # both cover sector N_b/2 - 1
    minus = set(range(0, math.ceil(X[-1])))
    plus = set(range(math.floor(X[1]), nb))
    assert nb // 2 - 1 in minus & plus
    new_plus = plus - minus
    gi = len(minus) * w[-1] + len(new_plus) * w[1]
    mask = sum(1 << k for k in minus | plus)
    swapped = (len(minus) - 1) * w[-1] + len(plus) * w[1]
    assert np.abs(gi - swapped).max() > 1e-3

    o0, _, masks, _ = oracle.fp64(oracle.Problem(g, prm, None), pixels=[(c, c)])
    assert int(masks[0, 0]) == mask
    np.testing.assert_allclose(o0[0, :3], gi, rtol=1e-12, atol=1e-15)
    assert o0[0, 3] == 1.0 - len(minus | plus) / nb
    r0, _, rmask = oracle.fp32(oracle.Problem(g, prm, None), pixels=[(c, c)])
    assert int(rmask[0, 0]) == mask
    np.testing.assert_allclose(r0[0, :3], gi, atol=2e-6)


def test_two_overlapping_samples_credit_the_nearer_first():
    """Section 3.3: samples are taken near to far and a sector's indirect light comes from the
    first sample that occludes it.  Two samples on the +omega side of slice 0 (steps 0 and 1)
    whose sector runs overlap in part: the far sample contributes only its sectors the near
    one left free.  Crediting the last sample, or both, gives a different GI."""
    W = H = 41
    fx = 20.5
    cam = scenegen.Camera(fx, fx, 20.5, 20.5)
    c = 20
    radius, ns, nb, t = 2.0, 4, 32, 0.5
    z = 3.0
    offs = G.sample_offsets(radius, fx, z, ns)
    dq = [int(np.rint(offs[0])), int(np.rint(offs[1]))]
    zq = [float(np.float32(2.6)), float(np.float32(2.2))]  # the values the depth plane holds
    nq = [np.array([-0.9, 0.0, 0.436], dtype=np.float32), np.array([-0.95, 0.0, 0.312], dtype=np.float32)]
    cq = [np.array([0.9, 0.1, 0.1], dtype=np.float32), np.array([0.1, 0.8, 0.3], dtype=np.float32)]
    depth = np.full((H, W), np.inf, dtype=np.float32)
    nrm = np.zeros((H, W, 4), dtype=np.float32)
    rad = np.zeros((H, W, 4), dtype=np.float32)
    depth[c, c] = z
    nrm[c, c, :3] = (0.0, 0.0, 1.0)
    for k in range(2):
        depth[c, c + dq[k]] = zq[k]
        nrm[c, c + dq[k], :3] = nq[k]
        rad[c, c + dq[k], :3] = cq[k]
    g = scenegen.GBuffer(depth, nrm, rad, cam)
    prm = Params(num_slices=1, steps_per_side=ns, radius=radius, thickness=t, sector_count=nb)

    n_p = np.array([0.0, 0.0, 1.0])
    p, v, s, gamma = G.frame(cam, c, c, z, n_p, np.float32(1.0), np.float32(0.0))
    masks, weights = [], []
    for k in range(2):
        sf = G.unproject(cam, c + dq[k] + 0.5, c + 0.5, zq[k])
        l = sf - p
        sb = sf + t * p / np.linalg.norm(p)
        hf = math.acos(np.dot(l, v) / np.linalg.norm(l))
        hb = math.acos(np.dot(sb - p, v) / np.linalg.norm(sb - p))
        A, B = sorted([G.sector_coord(hf, gamma, nb), G.sector_coord(hb, gamma, nb)])
        masks.append(G.half_covered_mask(A, B, nb))
        lh = l / np.linalg.norm(l)
        weights.append(max(0.0, float(np.dot(n_p, lh))) * max(0.0, -float(np.dot(nq[k].astype(np.float64), lh))))
    m0, m1 = masks
    pop = lambda m: bin(m).count("1")
    # the scene does what the test needs: partial overlap, both samples lit
    assert pop(m0 & m1) >= 2 and pop(m1 & ~m0) >= 2 and pop(m0 & ~m1) >= 2
    assert min(weights) > 0.1
    c64 = [x.astype(np.float64) for x in cq]
    first = (pop(m0) * weights[0] * c64[0] + pop(m1 & ~m0) * weights[1] * c64[1]) / nb
    last = (pop(m0 & ~m1) * weights[0] * c64[0] + pop(m1) * weights[1] * c64[1]) / nb
    both = (pop(m0) * weights[0] * c64[0] + pop(m1) * weights[1] * c64[1]) / nb
    assert np.abs(first - last).max() > 1e-2 and np.abs(first - both).max() > 1e-2

    o0, _, m, _ = oracle.fp64(oracle.Problem(g, prm, None), pixels=[(c, c)])
    assert int(m[0, 0]) == m0 | m1
    np.testing.assert_allclose(o0[0, :3], first, rtol=1e-12, atol=1e-15)
    assert abs(o0[0, 3] - (1.0 - pop(m0 | m1) / nb)) < 1e-15
    r0, _, rm = oracle.fp32(oracle.Problem(g, prm, None), pixels=[(c, c)])
    assert int(rm[0, 0]) == m0 | m1
    np.testing.assert_allclose(r0[0, :3], first, atol=2e-6)


# --- monotonicity (Section 3.1: samples only add occlusion; thicker slabs cover more) ---------

def _subset(a, b):
    return np.all((a & ~b) == 0)


def test_masks_monotone_in_samples():
    """N_s -> 2 N_s + 1 with zero noise reads a superset of the same step offsets."""
    g = scenegen.render(21, 40, 32, 8, 3)
    for fn in (oracle.fp64, oracle.fp32):
        m_a = fn(oracle.Problem(g, Params(num_slices=3, steps_per_side=5, radius=2.5, thickness=0.4), None))[2]
        m_b = fn(oracle.Problem(g, Params(num_slices=3, steps_per_side=11, radius=2.5, thickness=0.4), None))[2]
        assert _subset(m_a, m_b)
        assert np.count_nonzero(m_b) > np.count_nonzero(m_a) > 0


def test_masks_monotone_in_thickness():
    g = scenegen.render(22, 40, 32, 8, 3)
    prev = None
    for t in (0.05, 0.2, 0.6, 2.0, INF):
        m = oracle.fp64(oracle.Problem(g, Params(num_slices=2, steps_per_side=8, thickness=t), scenegen.ign_table()))[2]
        if prev is not None:
            assert _subset(prev, m)
        prev = m


# --- ambient cones (Section 3.2) ------------------------------------------------------------

def test_constant_environment_ambient_is_L_times_visibility():
    """Band-0 SH only: every cone sees the same radiance L = c00 Y00, and the unoccluded
    sector counts over all cones sum to N_b - popc(b), so ambient = L * AO."""
    g = scenegen.render(31, 36, 30, 8, 2)
    sh = np.zeros((9, 3), dtype=np.float32)
    sh[0] = (0.8, 0.5, 0.3)
    prm = Params(num_slices=3, steps_per_side=6, ambient_cones=4)
    o0, o1, _, _ = oracle.fp64(oracle.Problem(g, prm, scenegen.ign_table(), sh))
    L = sh[0].astype(np.float64) * 0.5 * math.sqrt(1.0 / math.pi)
    geo = np.isfinite(g.depth.ravel())
    np.testing.assert_allclose(o1[geo, :3], o0[geo, 3:4] * L[None, :], rtol=1e-12, atol=1e-14)
    r0, r1, _ = oracle.fp32(oracle.Problem(g, prm, scenegen.ign_table(), sh))
    np.testing.assert_allclose(r1[geo, :3], r0[geo, 3:4] * L[None, :], atol=2e-6)


def test_linear_environment_ambient_closed_form():
    """Unoccluded pixel on the optical axis facing the camera: gamma = 0 on every slice and the
    N_a = 4 cone directions average to cos(pi/8)+cos(3pi/8) over 2 times v.  With a band-1 SH
    the ambient is linear in direction: L = c00 Y00 + c1 sqrt(3/4pi) (R v)."""
    W = H = 33
    g = scenegen.hand_quad_over_sky(W, H, depth=3.0, x0=0, x1=W, y0=0, y1=H)
    th = math.radians(20.0)
    R = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]], dtype=np.float32)
    g.camera.view_to_world = R
    sh = np.zeros((9, 3), dtype=np.float32)
    sh[0] = (0.7, 0.6, 0.5)
    sh[1] = (0.10, -0.05, 0.0)   # y
    sh[2] = (0.05, 0.10, -0.1)   # z
    sh[3] = (-0.1, 0.0, 0.08)    # x
    prm = Params(num_slices=4, steps_per_side=5, radius=1.0, ambient_cones=4)
    c = W // 2
    o0, o1, masks, _ = oracle.fp64(oracle.Problem(g, prm, None, sh), pixels=[(c, c)])
    assert np.all(masks == 0)
    k = (math.cos(math.pi / 8) + math.cos(3 * math.pi / 8)) / 2.0
    wv = R.astype(np.float64) @ np.array([0.0, 0.0, 1.0]) * k
    c0 = 0.5 * math.sqrt(1 / math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    s64 = sh.astype(np.float64)
    expect = s64[0] * c0 + c1 * (s64[1] * wv[1] + s64[2] * wv[2] + s64[3] * wv[0])
    np.testing.assert_allclose(o1[0, :3], expect, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("func", ["z2", "x2-y2"])
def test_quadratic_environment_ambient_is_the_cone_average(func):
    """Band-2 SH coefficients that represent a known quadratic function f of the world direction:
    the ambient term must be the average of f over the cone directions.  f = z^2 = 1/3 + (2/3)
    P2(z) (Legendre), i.e. c00 = 2 sqrt(pi)/3 and c20 = (4/3) sqrt(pi/5); f = x^2 - y^2, the
    projection 4 sqrt(pi/15) onto Y22.  Unoccluded pixel on the optical axis facing the camera,
    view-to-world rotated 20 degrees about x: gamma = 0, cone k of slice i points along
    cos(th_k) v + sin(th_k) s_i, th_k = -pi/2 + (k + 1/2) pi / N_a (Section 3.2), each cone
    weighted 1/N_a."""
    W = H = 33
    g = scenegen.hand_quad_over_sky(W, H, depth=3.0, x0=0, x1=W, y0=0, y1=H)
    th = math.radians(20.0)
    R = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]], dtype=np.float32)
    g.camera.view_to_world = R
    sh = np.zeros((9, 3), dtype=np.float32)
    if func == "z2":
        sh[0] = 2.0 * math.sqrt(math.pi) / 3.0
        sh[6] = 4.0 / 3.0 * math.sqrt(math.pi / 5.0)
        f = lambda w: w[2] * w[2]  # noqa: E731
    else:
        sh[8] = 4.0 * math.sqrt(math.pi / 15.0)
        f = lambda w: w[0] * w[0] - w[1] * w[1]  # noqa: E731
    nd, na = 4, 4
    prm = Params(num_slices=nd, steps_per_side=5, radius=1.0, ambient_cones=na)
    c = W // 2
    o0, o1, masks, _ = oracle.fp64(oracle.Problem(g, prm, None, sh), pixels=[(c, c)])
    assert np.all(masks == 0)
    Rd = R.astype(np.float64)
    v = np.array([0.0, 0.0, 1.0])
    expect = 0.0
    for i in range(nd):
        cphi, sphi = G.slice_dir(i, nd)
        _, _, s_i, gamma = G.frame(g.camera, c, c, 3.0, v, cphi, sphi)
        assert abs(gamma) < 1e-12
        for k in range(na):
            t = -math.pi / 2 + (k + 0.5) * math.pi / na
            expect += f(Rd @ (math.cos(t) * v + math.sin(t) * s_i)) / (nd * na)
    # the sample's FP32 rounding of the coefficients is the only difference from f itself
    np.testing.assert_allclose(o1[0, :3], expect, rtol=2e-7, atol=1e-12)
    r0, r1, _ = oracle.fp32(oracle.Problem(g, prm, None, sh), pixels=[(c, c)])
    np.testing.assert_allclose(r1[0, :3], expect, atol=2e-6)


def test_ambient_cones_follow_the_projected_normal():
    """With a tilted centre normal, each slice's cones are centred on its own projected normal:
    cone k of slice i points at gamma_i - pi/2 + (k + 1/2) pi / N_a from v (Section 3.2, Eq. 4
    frame), gamma_i = atan2(n.s_i, n.v).  A lone pixel over sky (no occlusion) with the SH
    coefficients of f = z + z^2 (z projects onto Y10 with sqrt(4 pi / 3); z^2 as above): the
    ambient term is f averaged over those directions in world space.  The linear part is what
    sees gamma: the cones are evenly spaced over a half circle, so the mean of any quadratic in
    (cos, sin) over them does not depend on gamma, while their mean direction is proportional to
    cos(gamma) v + sin(gamma) s.  A wrong sign or a missing gamma offset fails this."""
    W = H = 33
    c = W // 2
    g = scenegen.hand_quad_over_sky(W, H, depth=3.0, x0=c, x1=c + 1, y0=c, y1=c + 1)
    n = np.array([0.45, -0.30, 0.0], dtype=np.float64)
    n[2] = math.sqrt(1.0 - n[0] ** 2 - n[1] ** 2)
    g.normal[c, c, :3] = n.astype(np.float32)
    th = math.radians(20.0)
    R = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]], dtype=np.float32)
    g.camera.view_to_world = R
    sh = np.zeros((9, 3), dtype=np.float32)
    sh[0] = 2.0 * math.sqrt(math.pi) / 3.0
    sh[2] = math.sqrt(4.0 * math.pi / 3.0)
    sh[6] = 4.0 / 3.0 * math.sqrt(math.pi / 5.0)
    nd, na = 4, 8
    prm = Params(num_slices=nd, steps_per_side=5, radius=1.0, ambient_cones=na, sector_count=64)
    o0, o1, masks, _ = oracle.fp64(oracle.Problem(g, prm, None, sh), pixels=[(c, c)])
    assert np.all(masks == 0)
    Rd = R.astype(np.float64)
    nf = g.normal[c, c, :3].astype(np.float64)
    expect, gammas = 0.0, []
    for i in range(nd):
        cphi, sphi = G.slice_dir(i, nd)
        _, v, s_i, gamma = G.frame(g.camera, c, c, 3.0, nf, cphi, sphi)
        gammas.append(gamma)
        for k in range(na):
            t = gamma - math.pi / 2 + (k + 0.5) * math.pi / na
            w = Rd @ (math.cos(t) * v + math.sin(t) * s_i)
            expect += (w[2] + w[2] * w[2]) / (nd * na)
    assert min(abs(x) for x in gammas) > 0.05  # every slice's frame is rotated
    np.testing.assert_allclose(o1[0, :3], expect, rtol=2e-7, atol=1e-12)
    r0, r1, _ = oracle.fp32(oracle.Problem(g, prm, None, sh), pixels=[(c, c)])
    np.testing.assert_allclose(r1[0, :3], expect, atol=2e-6)


# --- the binary32 replica against the FP64 oracle on a seeded frame ---------------------------

def test_replica_ambient_form_is_the_sh_sum():
    """The binary32 replica weights its ambient cones against the SH environment written once per
    launch as a quadratic form of the view-space direction, b.a + a^T Q a (Section 3.2's ambient
    light; the FP64 oracle evaluates the nine basis functions instead).  For random rotations,
    random coefficients and random unit directions the form must equal the 3-band real SH sum of
    the world direction R a, evaluated here from the basis definitions (Y00 = 1/(2 sqrt(pi)),
    Y1m = sqrt(3/(4 pi)) (y, z, x), Y2m = sqrt(15/pi)/2 (xy, yz, xz), sqrt(5/pi)/4 (3z^2 - 1),
    sqrt(15/pi)/4 (x^2 - y^2)), to the binary32 rounding of the coefficients.  A dropped constant
    term, a wrong band-2 factor or an unrotated direction fails it."""
    rng = np.random.default_rng(41)
    c0, c1 = 0.5 * math.sqrt(1.0 / math.pi), math.sqrt(3.0 / (4.0 * math.pi))
    c2, c3, c4 = 0.5 * math.sqrt(15.0 / math.pi), 0.25 * math.sqrt(5.0 / math.pi), 0.25 * math.sqrt(15.0 / math.pi)
    for trial in range(8):
        R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        sh = rng.uniform(-1.0, 1.0, size=(9, 3))
        R32, sh32 = R.astype(np.float32), sh.astype(np.float32)
        b, q = oracle.ambient_form32(R32, sh32)
        a = rng.normal(size=(200, 3))
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        w = a @ R32.astype(np.float64).T
        x, y, z = w[:, 0], w[:, 1], w[:, 2]
        Y = np.stack([np.full_like(x, c0), c1 * y, c1 * z, c1 * x, c2 * x * y, c2 * y * z,
                      c3 * (3.0 * z * z - 1.0), c2 * x * z, c4 * (x * x - y * y)], axis=1)
        direct = Y @ sh32.astype(np.float64)  # [200, 3]
        for ch in range(3):
            Q = q[ch].astype(np.float64)
            form = (a @ b[ch].astype(np.float64) + Q[0] * a[:, 0] ** 2 + Q[1] * a[:, 1] ** 2 + Q[2] * a[:, 2] ** 2
                    + 2.0 * (Q[3] * a[:, 0] * a[:, 1] + Q[4] * a[:, 0] * a[:, 2] + Q[5] * a[:, 1] * a[:, 2]))
            assert np.abs(form - direct[:, ch]).max() < 2e-6, (trial, ch)


def test_replica_vs_fp64_on_256():
    w = scenegen.workload_256()
    prob = oracle.Problem(w.gbuf, w.params, w.noise)
    o0, o1, m64, margin, ratio = oracle.fp64(prob, ratio=True)
    r0, r1, m32 = oracle.fp32(prob)
    same = np.all(m64 == m32, axis=1)
    diff = m64 != m32
    assert np.all(ratio[diff] <= 1.0)
    assert same.mean() > 0.99
    assert np.abs(r0[same] - o0[same]).max() < 1e-5


def test_temporal_noise_tables_vary_and_stay_in_range():
    base = scenegen.ign_table(0)
    seen = set()
    for f in range(8):
        t = scenegen.ign_table(f)
        assert t.shape == (16, 2) and np.all(t >= 0.0) and np.all(t < 1.0)
        # xi_s = frac(xi_phi + 1/2)
        np.testing.assert_allclose((t[:, 0].astype(np.float64) + 0.5) % 1.0, t[:, 1], atol=1e-6)
        seen.add(t.tobytes())
    assert len(seen) == 8 and np.array_equal(base, scenegen.ign_table(64))


@pytest.mark.parametrize("seed,kw", [
    (28, dict(num_slices=2, steps_per_side=23, radius=3.0, step_mode=1, sector_count=128)),
    (15, dict(num_slices=3, steps_per_side=12, radius=2.0, sector_count=128, hit_rule=1)),
    (15, dict(num_slices=3, steps_per_side=12, radius=2.0, sector_count=64, hit_rule=1)),
])
def test_binary32_flips_lie_within_the_error_bound(seed, kw):
    """Where the replica and the FP64 oracle disagree on a sector, the FP64 decision lies within
    the binary32 error bound of its endpoints from its boundary.  The bound is what makes this
    checkable at N_b = 128: a sample elevation taken as acos of a cosine within rounding of +-1
    is only known to ~sqrt(2 eps) rad, so some flips lie farther than 1e-3 sector units from
    their boundary, while the bound stays far below a sector for ordinary samples."""
    H, W = (180, 320) if seed == 28 else (150, 200)
    g = scenegen.render(seed, W, H, 8, 3)
    prm = Params(**kw)
    prob = oracle.Problem(g, prm, scenegen.ign_table())
    _, _, m32 = oracle.fp32(prob)
    _, _, m64, margin, ratio = oracle.fp64(prob, ratio=True)
    diff = (m64 != m32).any(axis=2) if m64.ndim == 3 else m64 != m32
    assert diff.sum() >= 1
    assert np.all(ratio[diff] <= 1.0), ratio[diff].max()
    if prm.sector_count == 128 and prm.hit_rule == 1:
        assert margin[diff].max() > 1e-3  # a flat 1e-3 sector tolerance would reject these
    # not vacuous: most slices have every decision well outside its bound
    assert np.mean(ratio <= 1.0) < 0.15


@pytest.mark.parametrize("seed,W,H,kw", [
    (28, 320, 180, dict(num_slices=2, steps_per_side=23, radius=3.0, step_mode=1, sector_count=128)),
    (17, 200, 150, dict(num_slices=3, steps_per_side=12, radius=2.0, thickness=0.1, thickness_slope=0.05)),
    (1, 256, 256, dict(num_slices=4, steps_per_side=8, sector_count=64, hit_rule=1)),
    (3, 3840, 2160, None),  # the 4K workload (FP16 normal/radiance, 4 cones) on 1500 sampled pixels
])
def test_binary32_endpoints_within_the_error_bound(seed, W, H, kw):
    """Every sector coordinate the replica computes (front and back, before clamping) lies within
    the FP64 oracle's binary32 error bound of the FP64 value, over every sample of a frame, and the
    bound stays well below a sector for the median sample."""
    if kw is None:
        w = scenegen.workload_4k()
        g, prm, noise, sh = w.gbuf, w.params, w.noise, w.sh
        rng = np.random.default_rng(4)
        pixels = np.stack([rng.integers(0, W, 1500), rng.integers(0, H, 1500)], 1).astype(np.int32)
    else:
        g = scenegen.render(seed, W, H, 8, 3)
        prm, noise, sh, pixels = Params(**kw), scenegen.ign_table(), None, None
    e32, e64 = oracle.endpoint_trace(oracle.Problem(g, prm, noise, sh), pixels)
    n = 0
    for k in range(2):
        x32 = e32[..., k].astype(np.float64)
        x64, bound = e64[..., k], e64[..., 2 + k]
        ok = np.isfinite(x32) & np.isfinite(x64)
        n += ok.sum()
        assert np.all(np.abs(x32[ok] - x64[ok]) <= bound[ok]), np.max(np.abs(x32[ok] - x64[ok]) / bound[ok])
        assert np.median(bound[ok]) < 0.05 * prm.sector_count / 32
    assert n > 100000


# --- the decision-forced FP64 evaluation (GPU gate on every pixel) ----------------------------

FORCED_CASES = [
    (1, 256, 256, dict(num_slices=4, steps_per_side=8, radius=2.0, thickness=0.5), True),
    (15, 64, 48, dict(num_slices=3, steps_per_side=12, sector_count=128, ambient_cones=8), True),
    (14, 33, 70, dict(num_slices=4, steps_per_side=10, sector_count=64, step_mode=1, ambient_cones=4), True),
    (16, 45, 37, dict(num_slices=2, steps_per_side=9, sector_count=128, thickness=INF, hit_rule=1), True),
    (10, 64, 48, dict(num_slices=2, steps_per_side=8, thickness=0.1, thickness_slope=0.05), False),
]


def _forced_problem(seed, W, H, kw, use_noise):
    g = scenegen.render(seed, W, H, 8, 3)
    prm = Params(**kw)
    sh = scenegen.sh_environment(7) if prm.ambient_cones else None
    return oracle.Problem(g, prm, scenegen.ign_table() if use_noise else None, sh), prm


@pytest.mark.parametrize("seed,W,H,kw,use_noise", FORCED_CASES)
def test_forced_evaluation_equals_free_running_fp64_where_decisions_agree(seed, W, H, kw, use_noise):
    """The forced evaluation takes the replica's sector run for every sample and keeps everything
    else in FP64 (Algorithm 1; Section 3.3 crediting).  Where every FP64 decision lies beyond its
    binary32 error bound the two decide alike, so there it must reproduce the free-running oracle
    to 1e-12; on every pixel its masks must be the replica's and its outputs within binary32
    rounding of the replica's (the same decisions, arithmetic in two precisions)."""
    prob, prm = _forced_problem(seed, W, H, kw, use_noise)
    e0, e1, em, _, ratio = oracle.fp64(prob, ratio=True)
    f0, f1, fm, _ = oracle.fp64(prob, forced=True)
    r0, r1, rm = oracle.fp32(prob)
    assert np.array_equal(fm, rm)
    same = (em == rm) if em.ndim == 2 else (em == rm).all(axis=2)
    clear = same.all(axis=1) & (ratio.min(axis=1) > 1.0)
    assert clear.mean() > 0.6
    assert np.abs(f0[clear] - e0[clear]).max() <= 1e-12
    assert np.abs(f1[clear] - e1[clear]).max() <= 1e-12
    assert np.abs(f0 - r0).max() <= 1e-5 and np.abs(f1 - r1).max() <= 1e-5
    # not vacuous where it matters: some pixels are not clear, and there the forced evaluation
    # follows the replica's decisions rather than the free-running oracle's
    if not clear.all():
        assert np.abs(f0[~clear] - r0[~clear]).max() <= 1e-5


def test_replica_runs_make_up_its_masks():
    """The per-sample runs the forced evaluation consumes are the replica's: OR-ing a slice's runs
    gives its mask, and every run lies inside [0, N_b]."""
    prob, prm = _forced_problem(15, 64, 48, dict(num_slices=3, steps_per_side=12, sector_count=128,
                                                 ambient_cones=8), True)
    runs = oracle.runs32(prob).astype(np.int64)
    _, _, rm = oracle.fp32(prob)
    lo, hi = runs[..., 0], runs[..., 1]
    assert np.all((hi <= lo) | ((lo >= 0) & (hi <= 128)))
    assert (hi > lo).sum() > 1000
    k = np.arange(128)
    cover = ((k >= lo[..., None]) & (k < hi[..., None])).any(axis=(2, 3))  # [n, N_d, 128]
    words = np.zeros(rm.shape, dtype=np.uint64)
    for w in range(2):
        bits = cover[..., 64 * w:64 * (w + 1)].astype(np.uint64) << np.arange(64, dtype=np.uint64)
        words[..., w] = np.bitwise_or.reduce(bits, axis=-1)
    assert np.array_equal(words, rm)


def test_forced_empty_runs_give_full_visibility():
    """Forcing every run empty leaves nothing occluded: AO = 1 and GI = 0 exactly, and with a
    constant (band-0) environment every cone sees its full sector share, so the ambient is the
    constant radiance c_00 Y_00 (Section 3.2)."""
    import ctypes
    g = scenegen.render(12, 40, 30, 8, 3)
    prm = Params(num_slices=3, steps_per_side=8, ambient_cones=4)
    sh = np.zeros((9, 3), dtype=np.float32)
    sh[0] = [0.9, 0.6, 0.3]
    prob = oracle.Problem(g, prm, scenegen.ign_table(), sh)
    xy = oracle.all_pixels(30, 40)
    n = len(xy)
    o0 = np.zeros((n, 4)); o1 = np.zeros((n, 4)); m = np.zeros((n, 3), dtype=np.uint64)
    runs = np.zeros((n, 3, 2, 8, 2), dtype=np.int16)
    rc = oracle.lib().orc64_pixels_ex(ctypes.byref(prob.c), n, xy.ctypes.data, o0.ctypes.data, o1.ctypes.data,
                                      m.ctypes.data, None, None, runs.ctypes.data, None, None)
    assert rc == 0
    assert np.all(m == 0) and np.all(o0[:, 3] == 1.0) and np.all(o0[:, :3] == 0.0)
    geo = np.isfinite(g.depth.reshape(-1)) & (g.depth.reshape(-1) > 0)
    expect = sh[0].astype(np.float64) * 0.5 * math.sqrt(1.0 / math.pi)
    np.testing.assert_allclose(o1[geo, :3], np.broadcast_to(expect, (geo.sum(), 3)), rtol=1e-12)
    bad = runs.copy()
    bad[0, 0, 0, 0] = (3, 200)  # a run beyond N_b is rejected
    assert oracle.lib().orc64_pixels_ex(ctypes.byref(prob.c), n, xy.ctypes.data, None, None, None, None, None,
                                        bad.ctypes.data, None, None) == 11


def test_results_do_not_depend_on_the_thread_count():
    """Pixels are independent; the OpenMP pixel loops must give the same bits on 1 thread and on
    all of them (outputs, masks, counters, runs)."""
    prob, prm = _forced_problem(14, 33, 70, dict(num_slices=4, steps_per_side=10, sector_count=64, step_mode=1,
                                                 ambient_cones=4), True)
    full = oracle.threads()
    try:
        res = []
        for t in (1, max(full, 2)):
            oracle.threads(t)
            res.append((oracle.fp32(prob, counts=True), oracle.fp64(prob, ratio=True), oracle.runs32(prob),
                        oracle.fp64(prob, forced=True)))
    finally:
        oracle.threads(full)
    (a32, a64, ar, af), (b32, b64, br, bf) = res
    for x, y in zip(a32[:3] + a64 + af, b32[:3] + b64 + bf):
        assert np.array_equal(x, y)
    assert a32[3] == b32[3] and np.array_equal(ar, br)


# --- the step offsets against the exact real-number step formula (Algorithm 1, R1, R19) --------

@pytest.mark.parametrize("step_mode,nd,ns,radius", [(0, 4, 32, 2.0), (1, 3, 17, 2.5), (0, 2, 5, 40.0)])
def test_step_offsets_are_the_nearest_pixels_of_the_exact_offsets(step_mode, nd, ns, radius):
    """Which pixel step j of side sigma reads is decided in binary32 (the GPU's decision, shared by
    both CPU programs).  Pinned here against the exact formula, evaluated independently in double
    precision from the inputs: offset o = (j + 1 + xi_s) r / (N_s + 1) (quadratic steps:
    r ((j + 1 + xi_s) / (N_s + 1))^2), r = R f_x / z, along sigma (cos phi_i, sin phi_i), phi_i =
    (i + xi_phi) pi / N_d, image y down in the direction table.  Every offset must be the nearest
    integer of the exact one per axis: within 1/2 pixel plus a rounding allowance of 1e-5 of the
    offset.  Using j instead of j + 1, dropping xi_s or flipping a side moves offsets by at least a
    step (tens of pixels here) and fails."""
    w = scenegen.workload_4k()
    prm = Params(nd, ns, radius, 0.5, step_mode=step_mode)
    prob = oracle.Problem(w.gbuf, prm, w.noise, None)
    H, W = w.gbuf.depth.shape
    rng = np.random.default_rng(21 + step_mode)
    xy = np.stack([rng.integers(0, W, 3000), rng.integers(0, H, 3000)], 1).astype(np.int32)
    st = oracle.step_offsets(prob, xy).astype(np.float64)          # [n, nd, 2, ns, 2]
    z = w.gbuf.depth[xy[:, 1], xy[:, 0]].astype(np.float64)
    geo = np.isfinite(z) & (z > 0)
    cls = (xy[:, 1] & 3) * 4 + (xy[:, 0] & 3)
    xi_phi = w.noise[cls, 0].astype(np.float64)
    xi_s = w.noise[cls, 1].astype(np.float64)
    r = np.minimum(np.float64(np.float32(radius)) * np.float64(w.gbuf.camera.fx) / np.where(geo, z, 1.0), 2.0 ** 20)
    j = np.arange(ns, dtype=np.float64)
    u = (j[None, :] + 1.0 + xi_s[:, None]) / (ns + 1)               # [n, ns]
    o = r[:, None] * (u * u if step_mode else u)
    phi = (np.arange(nd)[None, :] + xi_phi[:, None]) * math.pi / nd  # [n, nd]
    sigma = np.array([-1.0, 1.0])
    ex = sigma[None, None, :, None] * o[:, None, None, :] * np.cos(phi)[:, :, None, None]
    ey = sigma[None, None, :, None] * o[:, None, None, :] * np.sin(phi)[:, :, None, None]
    tol = 0.5 + 1e-5 * np.abs(o)[:, None, None, :] + 1e-6
    dx, dy = np.abs(st[..., 0] - ex), np.abs(st[..., 1] - ey)
    assert np.all(dx[geo] <= tol[geo]), dx[geo].max()
    assert np.all(dy[geo] <= tol[geo]), dy[geo].max()
    assert np.abs(st[geo]).max() > 50  # not vacuous: offsets of many pixels
