"""Seeded synthetic workloads shaped like the paper's 3DGS scenes and planner
query batches.  Both the CUDA path's tests/benchmark and the oracle consume
these arrays; the module holds none of the metric's arithmetic.

The paper evaluates on a reconstructed Stonehenge scene (about 200k splats,
Section III-A) and on real tabletop/room reconstructions; none of those is
available, so seeded stand-ins with the same structure are generated here:

  tiny_scene        2k Gaussians, uniform in a 2 m cube
  drone_scene       500k: 70 % flat splats on the walls of a 6x5x3 m room,
                    30 % in 40 isotropic clutter clusters
  tabletop_scene    1M: a 1.2x0.8 m table plane plus 25 object clusters
  apartment_scene   3M: a 12x8x2.7 m four-room flat (walls with door gaps)
                    plus furniture clusters
  tabletop_disks    the tabletop as a 2DGS scene: every Gaussian a disk (its
                    third scale zero, Section I)
  tabletop_points   the tabletop as a point cloud (every scale zero)

Queries are sphere batches laid out the way MPPI and RRT consume them
(Section II-D: (K, T, N_link); Section II-E: (N_batch, N_strides, N_links)),
and one ellipsoid per link of the same arm (arm_ellipsoids).

Conventions: float32 arrays; quaternions (w, x, y, z); scales are per-axis
standard deviations in metres; opacity in [0, 1]; sphere rows (cx, cy, cz, r).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "tiny_scene", "tiny_queries", "drone_scene", "drone_queries", "tabletop_scene",
    "arm_queries", "edge_queries", "trajectory_poses", "apartment_scene",
    "serving_requests", "random_quats", "matrix_to_quat", "ellipsoid_queries",
    "tabletop_disks", "tabletop_points", "arm_ellipsoids", "look_at", "scene_colors",
    "drone_terminal_cameras", "tabletop_cameras",
]


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def random_quats(rng, n):
    """Uniform random unit quaternions (normalised 4-D Gaussian samples)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def matrix_to_quat(R):
    """Rotation matrices [n,3,3] -> unit quaternions (w,x,y,z), Shepperd's method."""
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    q = np.zeros((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    diag = np.stack([R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], 1)
    choice = np.where(tr > diag.max(1), 3, diag.argmax(1))
    for k in range(4):
        m = choice == k
        if not m.any():
            continue
        Rm = R[m]
        if k == 3:
            s = np.sqrt(1.0 + tr[m]) * 2.0
            q[m, 0] = 0.25 * s
            q[m, 1] = (Rm[:, 2, 1] - Rm[:, 1, 2]) / s
            q[m, 2] = (Rm[:, 0, 2] - Rm[:, 2, 0]) / s
            q[m, 3] = (Rm[:, 1, 0] - Rm[:, 0, 1]) / s
        else:
            i, j, l = k, (k + 1) % 3, (k + 2) % 3
            s = np.sqrt(1.0 + Rm[:, i, i] - Rm[:, j, j] - Rm[:, l, l]) * 2.0
            q[m, 0] = (Rm[:, l, j] - Rm[:, j, l]) / s
            q[m, 1 + i] = 0.25 * s
            q[m, 1 + j] = (Rm[:, j, i] + Rm[:, i, j]) / s
            q[m, 1 + l] = (Rm[:, l, i] + Rm[:, i, l]) / s
    return q


def _pack(means, scales, quats, opacity):
    return {
        "means": np.ascontiguousarray(means, np.float32),
        "scales": np.ascontiguousarray(scales, np.float32),
        "quats": np.ascontiguousarray(quats, np.float32),
        "opacity": np.ascontiguousarray(opacity, np.float32),
    }


def _flat_splats(rng, n, origin, u, v, extent_u, extent_v, tangent_median, normal_median,
                 sigma_log=0.3):
    """n flat splats uniformly on the rectangle origin + [0,eu] u + [0,ev] v,
    normal axis (third scale) along u x v, random in-plane rotation."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    nrm = np.cross(u, v)
    a = rng.uniform(0, extent_u, n)
    b = rng.uniform(0, extent_v, n)
    means = np.asarray(origin)[None] + a[:, None] * u[None] + b[:, None] * v[None]
    th = rng.uniform(0, 2 * np.pi, n)
    t1 = np.cos(th)[:, None] * u[None] + np.sin(th)[:, None] * v[None]
    t2 = -np.sin(th)[:, None] * u[None] + np.cos(th)[:, None] * v[None]
    R = np.stack([t1, t2, np.broadcast_to(nrm, t1.shape)], axis=2)
    quats = matrix_to_quat(R)
    scales = np.stack([
        tangent_median * np.exp(sigma_log * rng.normal(size=n)),
        tangent_median * np.exp(sigma_log * rng.normal(size=n)),
        normal_median * np.exp(sigma_log * rng.normal(size=n))], axis=1)
    return means, scales, quats


def _clusters(rng, n, centres_lo, centres_hi, n_clusters, spread, log_median, log_sigma,
              z_floor=None, sizes=None):
    if sizes is None:
        sizes = rng.multinomial(n, np.full(n_clusters, 1.0 / n_clusters))
    centres = rng.uniform(centres_lo, centres_hi, size=(len(sizes), 3))
    spreads = np.broadcast_to(np.asarray(spread, np.float64), (len(sizes),))
    means = np.concatenate([c[None] + s * rng.normal(size=(k, 3))
                            for c, s, k in zip(centres, spreads, sizes)])
    if z_floor is not None:
        means[:, 2] = z_floor + np.abs(means[:, 2] - z_floor)
    m = means.shape[0]
    scales = np.exp(np.log(log_median) + log_sigma * rng.normal(size=(m, 3)))
    return means, scales, random_quats(rng, m)


# --------------------------------------------------------------- config 1
def tiny_scene(seed=1001, n=2000):
    """N Gaussians, means uniform in a 2 m cube, log-scales ~ N(ln 0.02, 0.5),
    uniform rotations, opacity = sigmoid(N(0, 1.5))."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.0, 2.0, size=(n, 3))
    scales = np.exp(np.log(0.02) + 0.5 * rng.normal(size=(n, 3)))
    return _pack(means, scales, random_quats(rng, n), _sigmoid(rng.normal(0, 1.5, n)))


def tiny_queries(seed=1001, q=256):
    """Spheres with centres uniform in the cube, radii uniform in [0.05, 0.2] m."""
    rng = np.random.default_rng(seed + 500)
    c = rng.uniform(0.0, 2.0, size=(q, 3))
    r = rng.uniform(0.05, 0.2, size=(q, 1))
    return np.ascontiguousarray(np.concatenate([c, r], 1), np.float32)


def ellipsoid_queries(seed, centres, semi_lo=0.03, semi_hi=0.2):
    """Ellipsoids (cx,cy,cz, qw,qx,qy,qz, a,b,c) at the given centres."""
    rng = np.random.default_rng(seed)
    q = centres.shape[0]
    quats = random_quats(rng, q)
    axes = rng.uniform(semi_lo, semi_hi, size=(q, 3))
    return np.ascontiguousarray(np.concatenate([centres, quats, axes], 1), np.float32)


# --------------------------------------------------------------- config 2
_ROOM = np.array([6.0, 5.0, 3.0])


def _box_faces(lo, hi):
    """The six inward-facing faces of an axis-aligned box as (origin, u, v, eu, ev)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    ex, ey, ez = hi - lo
    X, Y, Z = np.eye(3)
    return [
        (lo, X, Y, ex, ey),                          # floor, normal +z
        (np.array([lo[0], hi[1], hi[2]]), X, -Y, ex, ey),   # ceiling, normal -z
        (lo, Y, Z, ey, ez),                          # x = lo, normal +x
        (np.array([hi[0], hi[1], lo[2]]), -Y, Z, ey, ez),   # x = hi, normal -x
        (np.array([hi[0], lo[1], lo[2]]), -X, Z, ex, ez),   # y = lo, normal +y
        (np.array([lo[0], hi[1], lo[2]]), X, Z, ex, ez),    # y = hi, normal -y
    ]


def _surface_splats(rng, n, faces, tangent_median, normal_median):
    areas = np.array([f[3] * f[4] for f in faces])
    counts = rng.multinomial(n, areas / areas.sum())
    parts = [_flat_splats(rng, k, o, u, v, eu, ev, tangent_median, normal_median)
             for (o, u, v, eu, ev), k in zip(faces, counts) if k > 0]
    return tuple(np.concatenate([p[i] for p in parts]) for i in range(3))


def drone_scene(seed=1002, n=500_000):
    """A 6x5x3 m room: 70 % flat splats on the six faces (tangent scales
    median 3 cm, normal scale median 3 mm, log-sigma 0.3), 30 % in 40 clutter
    clusters (centres in the room shrunk by 0.5 m, spread 0.15 m, scales
    log N(ln 0.02, 0.5)); opacity sigmoid(N(0, 1.5))."""
    rng = np.random.default_rng(seed)
    n_surf = int(round(0.7 * n))
    m1, s1, q1 = _surface_splats(rng, n_surf, _box_faces(np.zeros(3), _ROOM), 0.03, 0.003)
    m2, s2, q2 = _clusters(rng, n - n_surf, 0.5, _ROOM - 0.5, 40, 0.15, 0.02, 0.5)
    means = np.concatenate([m1, m2])
    return _pack(means, np.concatenate([s1, s2]), np.concatenate([q1, q2]),
                 _sigmoid(rng.normal(0, 1.5, means.shape[0])))


def _random_walks(rng, n_walks, steps, lo, hi, speed=0.5, dt=0.1, jitter=0.15):
    """Smooth random walks reflected at the box walls: [n_walks, steps, 3]."""
    pos = rng.uniform(lo, hi, size=(n_walks, 3))
    vel = rng.normal(0.0, speed, size=(n_walks, 3))
    out = np.empty((n_walks, steps, 3))
    for t in range(steps):
        out[:, t] = pos
        vel += rng.normal(0.0, jitter, size=vel.shape)
        pos = pos + vel * dt
        low = pos < lo
        high = pos > hi
        pos = np.where(low, 2 * lo - pos, pos)
        pos = np.where(high, 2 * hi - pos, pos)
        vel = np.where(low | high, -vel, vel)
        pos = np.clip(pos, lo, hi)
    return out


def drone_queries(seed=1002, rollouts=1024, horizon=32, radius=0.15):
    """MPPI batch (K, T, 1): K rollouts of T steps of a drone sphere; rows are
    ordered rollout-major so a group of T consecutive rows is one rollout."""
    rng = np.random.default_rng(seed + 500)
    walks = _random_walks(rng, rollouts, horizon, np.full(3, 0.2), _ROOM - 0.2)
    c = walks.reshape(-1, 3)
    r = np.full((c.shape[0], 1), radius)
    return np.ascontiguousarray(np.concatenate([c, r], 1), np.float32)


# --------------------------------------------------------------- config 3
_TABLE = np.array([1.2, 0.8])
_ARM_BASE = np.array([0.0, -0.5, 0.0])


def tabletop_scene(seed=1003, n=1_000_000, n_clusters=25):
    """A 1.2x0.8 m table plane at z = 0 centred on the origin plus object
    clusters of 5-40k Gaussians each (spread 2-8 cm, resting on the table),
    scales log-normal with median 3.16 mm and log-sigma ln(10)/4 (95 % within
    1-10 mm).  Plane splats are flat (normal scale 0.3x) and face up."""
    rng = np.random.default_rng(seed)
    scale_cluster = n / 1_000_000
    while True:
        sizes = rng.integers(5_000, 40_001, n_clusters)
        sizes = np.maximum(1, (sizes * scale_cluster).astype(np.int64))
        if sizes.sum() <= 0.9 * n:
            break
    n_plane = n - int(sizes.sum())
    med, sl = 0.00316, np.log(10.0) / 4.0
    half = _TABLE / 2
    origin = np.array([-half[0], -half[1], 0.0])
    m1, s1, q1 = _flat_splats(rng, n_plane, origin, [1, 0, 0], [0, 1, 0], _TABLE[0], _TABLE[1],
                              med, 0.3 * med, sigma_log=sl)
    centres_lo = np.array([-half[0] + 0.1, -half[1] + 0.1, 0.0])
    centres_hi = np.array([half[0] - 0.1, half[1] - 0.1, 0.05])
    spreads = rng.uniform(0.02, 0.08, len(sizes))
    m2, s2, q2 = _clusters(rng, None, centres_lo, centres_hi, len(sizes), spreads, med, sl,
                           z_floor=0.0, sizes=sizes)
    means = np.concatenate([m1, m2])
    return _pack(means, np.concatenate([s1, s2]), np.concatenate([q1, q2]),
                 _sigmoid(rng.normal(0, 1.5, means.shape[0])))


_AXES = np.array([[0, 0, 1], [0, 1, 0], [0, 0, 1], [0, 1, 0], [0, 0, 1], [0, 1, 0], [0, 0, 1]],
                 np.float64)
_LINK = np.array([0.18, 0.20, 0.16, 0.16, 0.12, 0.10, 0.08])  # 1.0 m in total


def _axis_rot(axis, ang):
    """Rotation matrices [n,3,3] about a fixed unit axis by angles [n]."""
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    s, c = np.sin(ang)[:, None, None], np.cos(ang)[:, None, None]
    return np.eye(3)[None] + s * K[None] + (1 - c) * (K @ K)[None]


def _arm_spheres(joints, n_spheres=64):
    """Serial 7-joint chain from the arm base; returns sphere rows [n, 64, 4],
    spheres evenly spaced along the 1 m of links, radii 8 cm -> 2 cm."""
    n = joints.shape[0]
    R = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    p = np.broadcast_to(_ARM_BASE, (n, 3)).copy()
    pts = [p.copy()]
    for k in range(7):
        R = R @ _axis_rot(_AXES[k], joints[:, k])
        p = p + R[:, :, 2] * _LINK[k]
        pts.append(p.copy())
    pts = np.stack(pts, 1)                      # [n, 8, 3]
    cum = np.concatenate([[0.0], np.cumsum(_LINK)])
    s = np.linspace(0.0, cum[-1], n_spheres)
    idx = np.clip(np.searchsorted(cum, s, side="right") - 1, 0, 6)
    frac = (s - cum[idx]) / _LINK[idx]
    centres = pts[:, idx] + frac[None, :, None] * (pts[:, idx + 1] - pts[:, idx])
    radii = np.broadcast_to(np.linspace(0.08, 0.02, n_spheres), (n, n_spheres))
    return np.concatenate([centres, radii[..., None]], -1)


def _random_joints(rng, n):
    j = rng.uniform(-np.pi, np.pi, size=(n, 7))
    j[:, 0] = rng.uniform(0.2, np.pi - 0.2, n)  # base yaw: facing the table (+y)
    j[:, 1] = rng.uniform(0.2, 1.9, n)          # shoulder pitched over the table
    j[:, 3] = rng.uniform(-2.0, 2.0, n)
    return j


def tabletop_disks(seed=1003, n=1_000_000):
    """The tabletop with every Gaussian flattened into a 2DGS disk: the third
    scale (the plane splats' normal axis; a random axis of the cluster
    Gaussians) set to zero."""
    sc = tabletop_scene(seed, n)
    sc["scales"][:, 2] = 0.0
    return sc


def tabletop_points(seed=1003, n=1_000_000):
    """The tabletop's means as a point cloud: every scale zero."""
    sc = tabletop_scene(seed, n)
    sc["scales"][:] = 0.0
    return sc


def _arm_ellipsoids(joints):
    """One ellipsoid per link of the 7-joint chain: centred on the link's
    midpoint, its third axis along the link (semi-axis half the link plus the
    radius), the first two the link radius (8 cm at the base to 2 cm at the
    tip); rows [n, 7, 10]."""
    n = joints.shape[0]
    R = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    p = np.broadcast_to(_ARM_BASE, (n, 3)).copy()
    radii = np.linspace(0.08, 0.02, 7)
    rows = []
    for k in range(7):
        R = R @ _axis_rot(_AXES[k], joints[:, k])
        q = p + R[:, :, 2] * _LINK[k]
        semi = np.broadcast_to([radii[k], radii[k], _LINK[k] / 2 + radii[k]], (n, 3))
        rows.append(np.concatenate([(p + q) / 2, matrix_to_quat(R), semi], 1))
        p = q
    return np.stack(rows, 1)


def arm_ellipsoids(seed=1003, configs=32768):
    """Multi-link ellipsoid robot batch: configs x 7 link ellipsoids (one group
    of 7 rows per configuration); 229,376 rows by default."""
    rng = np.random.default_rng(seed + 900)
    e = _arm_ellipsoids(_random_joints(rng, configs))
    return np.ascontiguousarray(e.reshape(-1, 10), np.float32)


def arm_queries(seed=1003, configs=4096):
    """RRT/MPPI arm batch: configs x 64 link spheres, one group of 64 rows per
    configuration."""
    rng = np.random.default_rng(seed + 500)
    sph = _arm_spheres(_random_joints(rng, configs))
    return np.ascontiguousarray(sph.reshape(-1, 4), np.float32)


def edge_queries(seed=1003, edges=2048, strides=16, max_step=0.3):
    """RRT edge batch (N_batch, N_strides, N_links): each edge joins a random
    configuration to a neighbour at most max_step rad away per joint, checked at
    `strides` interpolated configurations of 64 spheres."""
    rng = np.random.default_rng(seed + 700)
    a = _random_joints(rng, edges)
    b = a + rng.uniform(-max_step, max_step, size=a.shape)
    t = np.linspace(0.0, 1.0, strides)
    q = a[:, None] + t[None, :, None] * (b - a)[:, None]
    sph = _arm_spheres(q.reshape(-1, 7))
    return np.ascontiguousarray(sph.reshape(-1, 4), np.float32)


# --------------------------------------------------------------- config 4
def trajectory_poses(seed=1004, trajectories=512, waypoints=64):
    """Differentiable batch: per-waypoint poses (t, w) [T*W, 6] along smooth
    curves over the table (heights 2-30 cm), the 8 body-frame sphere offsets
    (corners of a +-5 cm box) and the sphere radius 3 cm."""
    rng = np.random.default_rng(seed)
    half = _TABLE / 2
    p0 = np.concatenate([rng.uniform(-half, half, (trajectories, 2)),
                         rng.uniform(0.02, 0.3, (trajectories, 1))], 1)
    p1 = np.concatenate([rng.uniform(-half, half, (trajectories, 2)),
                         rng.uniform(0.02, 0.3, (trajectories, 1))], 1)
    s = np.linspace(0, 1, waypoints)[None, :, None]
    amp = rng.normal(0, 0.05, (trajectories, 1, 3))
    phase = rng.uniform(0, 2 * np.pi, (trajectories, 1, 3))
    t = p0[:, None] + s * (p1 - p0)[:, None] + amp * np.sin(2 * np.pi * s + phase)
    t[..., 2] = np.clip(t[..., 2], 0.02, 0.35)
    w0 = rng.normal(0, 0.6, (trajectories, 1, 3))
    w1 = rng.normal(0, 0.6, (trajectories, 1, 3))
    w = w0 + s * (w1 - w0)
    poses = np.concatenate([t, w], -1).reshape(-1, 6)
    corners = np.array([[x, y, z] for x in (-0.05, 0.05) for y in (-0.05, 0.05)
                        for z in (-0.05, 0.05)])
    return (np.ascontiguousarray(poses, np.float32), np.ascontiguousarray(corners, np.float32),
            0.03)


# --------------------------------------------------------------- config 5
_FLAT = np.array([12.0, 8.0, 2.7])


def _apartment_faces():
    faces = _box_faces(np.zeros(3), _FLAT)
    X, Y, Z = np.eye(3)
    h = _FLAT[2]
    # interior wall x = 6 (door gaps y in [1.5, 2.4] and [5.5, 6.4]) and
    # interior wall y = 4 (door gaps x in [2.5, 3.4] and [8.5, 9.4]); both sides
    for y0, y1 in ((0.0, 1.5), (2.4, 5.5), (6.4, 8.0)):
        faces.append((np.array([6.0, y0, 0.0]), Y, Z, y1 - y0, h))
        faces.append((np.array([6.0, y1, 0.0]), -Y, Z, y1 - y0, h))
    for x0, x1 in ((0.0, 2.5), (3.4, 8.5), (9.4, 12.0)):
        faces.append((np.array([x1, 4.0, 0.0]), -X, Z, x1 - x0, h))
        faces.append((np.array([x0, 4.0, 0.0]), X, Z, x1 - x0, h))
    return faces


def apartment_scene(seed=1005, n=3_000_000, n_clusters=120):
    """A 12x8x2.7 m flat with four rooms: 70 % flat splats on the outer and
    interior walls, floor and ceiling (config-2 surface law), 30 % in
    furniture clusters (config-2 cluster law)."""
    rng = np.random.default_rng(seed)
    n_surf = int(round(0.7 * n))
    m1, s1, q1 = _surface_splats(rng, n_surf, _apartment_faces(), 0.03, 0.003)
    lo = np.array([0.5, 0.5, 0.3])
    hi = _FLAT - np.array([0.5, 0.5, 1.2])
    m2, s2, q2 = _clusters(rng, n - n_surf, lo, hi, n_clusters, 0.15, 0.02, 0.5)
    means = np.concatenate([m1, m2])
    return _pack(means, np.concatenate([s1, s2]), np.concatenate([q1, q2]),
                 _sigmoid(rng.normal(0, 1.5, means.shape[0])))


def serving_requests(seed=1007, count=1000, q_lo=16, q_hi=262_144, mean_interarrival_s=1e-3,
                     n_scenes=2):
    """Poisson-arriving requests: arrival time, scene id, n_sigma ~ U[0, 2] and
    a batch of spheres (random walks inside the flat, radii U[0.02, 0.2]) whose
    size is log-uniform in [q_lo, q_hi]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_interarrival_s, count)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(np.log(q_lo), np.log(q_hi), count)).astype(np.int64)
    out = []
    for k in range(count):
        q = int(sizes[k])
        steps = 16 if q >= 16 else q
        walks = _random_walks(rng, (q + steps - 1) // steps, steps, np.full(3, 0.2), _FLAT - 0.2)
        c = walks.reshape(-1, 3)[:q]
        r = rng.uniform(0.02, 0.2, (q, 1))
        out.append({
            "arrival": float(arrivals[k]),
            "scene": int(rng.integers(0, n_scenes)),
            "nsigma": float(rng.uniform(0.0, 2.0)),
            "spheres": np.ascontiguousarray(np.concatenate([c, r], 1), np.float32),
        })
    return out


# ------------------------------------------------------- rendering inputs
def look_at(eye, target, up=(0.0, 0.0, 1.0), f=100.0, width=128, height=128) -> np.ndarray:
    """Camera row (16 float32: world-to-camera R row-major, t, fx, fy, cx, cy)
    at `eye` looking at `target`: camera z along the view direction, x to the
    right, y down the image rows, principal point at the image centre."""
    eye = np.asarray(eye, np.float64)
    zc = np.asarray(target, np.float64) - eye
    zc /= np.linalg.norm(zc)
    xc = np.cross(zc, np.asarray(up, np.float64))
    xc /= np.linalg.norm(xc)
    yc = np.cross(zc, xc)
    R = np.stack([xc, yc, zc])
    t = -R @ eye
    return np.concatenate([R.ravel(), t, [f, f, width / 2.0, height / 2.0]]).astype(np.float32)


def scene_colors(scene, seed=1100) -> np.ndarray:
    """Per-Gaussian RGB in [0, 1] (view-independent colour, the degree-0 part
    of 3DGS appearance): a smooth function of position plus noise, so images
    have structure."""
    rng = np.random.default_rng(seed)
    m = np.asarray(scene["means"], np.float64)
    phase = rng.uniform(0, 2 * np.pi, 3)
    freq = rng.uniform(3.0, 9.0, 3)
    base = 0.5 + 0.35 * np.sin(m * freq[None] + phase[None])
    return np.ascontiguousarray(np.clip(base + rng.normal(0, 0.05, m.shape), 0, 1), np.float32)


def drone_terminal_cameras(seed=1002, rollouts=256, horizon=32, width=128, height=128, fov_deg=90.0):
    """Cameras at the terminal states of drone MPPI rollouts in the room
    (Section II-D: the terminal state of each rollout is rendered), looking
    along the last step's horizontal heading: [rollouts, 16] float32."""
    q = drone_queries(seed, rollouts=rollouts, horizon=horizon).reshape(rollouts, horizon, 4)
    eye = q[:, -1, :3].astype(np.float64)
    head = eye - q[:, -2, :3]
    head[:, 2] = 0.0
    nrm = np.linalg.norm(head, axis=1)
    head[nrm < 1e-6] = (1.0, 0.0, 0.0)
    head /= np.linalg.norm(head, axis=1, keepdims=True)
    f = 0.5 * width / np.tan(np.radians(fov_deg) / 2)
    return np.stack([look_at(e, e + h, f=f, width=width, height=height) for e, h in zip(eye, head)])


def tabletop_cameras(seed=1101, views=256, width=128, height=128, fov_deg=60.0):
    """Cameras on a hemisphere of radius 0.8-1.4 m around the table centre,
    looking at points on the table: [views, 16] float32."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0, 2 * np.pi, views)
    el = rng.uniform(np.radians(20), np.radians(70), views)
    r = rng.uniform(0.8, 1.4, views)
    eye = np.stack([r * np.cos(el) * np.cos(az), r * np.cos(el) * np.sin(az), r * np.sin(el)], 1)
    tgt = np.c_[rng.uniform(-0.3, 0.3, (views, 2)), np.zeros(views)]
    f = 0.5 * width / np.tan(np.radians(fov_deg) / 2)
    return np.stack([look_at(e, t, f=f, width=width, height=height) for e, t in zip(eye, tgt)])
