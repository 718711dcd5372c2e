"""Seeded synthetic phantoms and acquisition set-ups.

Input generation only: triangle meshes, media tables, point-scatterer clouds, probe and image
descriptors.  This module holds none of the method's arithmetic (no transport, pulse,
beamforming or derivative); both the CUDA path and the CPU oracle consume what it returns.

Units are SI (m, s, Hz, kg/m^3); attenuation is in dB/cm/MHz.  The parameter vector is
``theta = [c_0, rho_0, alpha_0, ..., c_{M-1}, rho_{M-1}, alpha_{M-1}, A_s, f0]`` with medium 0
the one the probe sits in.  Triangles carry ``(m_front, m_back)``: the front side is the one the
normal ``(v1 - v0) x (v2 - v0)`` points to; closed regions have outward normals, so
``m_front`` is the surrounding medium and ``m_back`` the region's own.

Workloads (the paper prints no scene data, so every one is synthetic and seeded):

* ``two_layer`` -- water over a tissue slab with a flat interface at 20 mm (a closed box
  x, y in +-20 mm, z in [20, 40] mm, 12 triangles); 64 elements, 0.3 mm pitch, 5 MHz, 60 %
  bandwidth, 40 MHz, 2048 samples, one unsteered plane wave, 1e4 rays per element, at most
  4 interactions, 128 x 1024 pixel B-mode.
* ``inclusions`` -- a 40 x 40 x 60 mm soft-tissue block holding 12 non-overlapping,
  randomly oriented ellipsoids (semi-axes U[2, 6] mm, 65 x 130 tessellation, 16,640 triangles
  each, 199,680 in total; c ~ U[1450, 1650], rho ~ U[950, 1150], alpha ~ U[0.3, 1.0]) plus 1e5
  point scatterers uniform in the block with N(0, 1) amplitudes and radius 0.1 mm; 128
  elements, 16 plane waves over -15..15 degrees, 7813 rays per element (1e6 per transmit), at
  most 8 interactions, 4096 samples, 256 x 1024 B-mode.
* ``differentiation`` -- the inclusion scene with one unsteered plane wave, at most 4
  interactions and 782 rays per element (1e5 per transmit); the target parameters are the
  reference ones scaled by (1 +- 5 %).
* ``slab_scatterers`` -- the two-layer slab with 1000 scatterers inside the slab (a small
  differentiation case with 8 parameters).
* ``hollow_cylinder`` -- a tube of outer radius R = 5 mm (wall 1 mm) whose axis runs along the
  elevation direction at 15 mm depth, in scattering tissue; the lumen holds a fluid without
  scatterers.  ``dtris_dR`` is the vertex tangent of the radius (both surfaces move outward
  with R, the wall thickness fixed).
"""
from __future__ import annotations

import math

import numpy as np

MM = 1e-3
DEG = math.pi / 180.0


# --------------------------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------------------------
def box_mesh(lo, hi):
    """12 triangles of an axis-aligned box with outward normals; returns (12, 9)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float64)
    quads = [(0, 3, 2, 1),  # z = z0, normal -z
             (4, 5, 6, 7),  # z = z1, normal +z
             (0, 1, 5, 4),  # y = y0, normal -y
             (2, 3, 7, 6),  # y = y1, normal +y
             (1, 2, 6, 5),  # x = x1, normal +x
             (0, 4, 7, 3)]  # x = x0, normal -x
    tris = []
    for a, b, c, d in quads:
        tris.append(np.concatenate([v[a], v[b], v[c]]))
        tris.append(np.concatenate([v[a], v[c], v[d]]))
    return np.asarray(tris)


def ellipsoid_mesh(center, semi, rot, n_lat=65, n_lon=130):
    """Closed UV-tessellated ellipsoid with outward normals: 2 * n_lon * (n_lat - 1) triangles."""
    theta = np.linspace(0.0, math.pi, n_lat + 1)
    phi = np.linspace(0.0, 2.0 * math.pi, n_lon + 1)[:-1]
    unit = np.stack([np.sin(theta)[:, None] * np.cos(phi)[None, :],
                     np.sin(theta)[:, None] * np.sin(phi)[None, :],
                     np.cos(theta)[:, None] * np.ones_like(phi)[None, :]], axis=-1)
    world = (unit * np.asarray(semi)[None, None, :]) @ np.asarray(rot).T + np.asarray(center)[None, None, :]
    j = np.arange(n_lon)
    j1 = (j + 1) % n_lon
    top = np.broadcast_to(world[0, 0], (n_lon, 3))
    bot = np.broadcast_to(world[n_lat, 0], (n_lon, 3))
    caps = [np.concatenate([top, world[1, j], world[1, j1]], axis=1),
            np.concatenate([bot, world[n_lat - 1, j1], world[n_lat - 1, j]], axis=1)]
    i = np.arange(1, n_lat - 1)
    a = world[i][:, j]
    b = world[i][:, j1]
    c = world[i + 1][:, j]
    d = world[i + 1][:, j1]
    band = np.stack([np.concatenate([a, c, d], axis=-1), np.concatenate([a, d, b], axis=-1)], axis=2)
    t = np.concatenate(caps + [band.reshape(-1, 9)], axis=0).copy()
    # orient outward: normal . (centroid - centre) > 0
    v0, v1, v2 = t[:, 0:3], t[:, 3:6], t[:, 6:9]
    n = np.cross(v1 - v0, v2 - v0)
    out = np.einsum("ij,ij->i", n, (v0 + v1 + v2) / 3.0 - np.asarray(center)[None, :])
    flip = out < 0
    t[flip] = np.concatenate([v0[flip], v2[flip], v1[flip]], axis=1)
    return t


def tube_mesh(radius, zc, half_len, n_phi, n_y, outward=True):
    """Open cylinder of the given radius around the axis x = 0, z = zc (along y): n_phi x n_y
    quads, two triangles each, normals pointing away from the axis (outward) or toward it.
    Returns (tris (2 n_phi n_y, 9), radial unit vector of every vertex (same shape)); quad
    (i, j) (azimuth i, along-axis j) gives triangles 2 (i n_y + j) and 2 (i n_y + j) + 1."""
    phi = np.linspace(0.0, 2.0 * np.pi, n_phi + 1)[:-1]
    ys = np.linspace(-half_len, half_len, n_y + 1)
    a0, a1 = np.repeat(phi, n_y), np.repeat(np.roll(phi, -1), n_y)
    y0, y1 = np.tile(ys[:-1], n_phi), np.tile(ys[1:], n_phi)

    def point(a, y):
        return np.stack([radius * np.cos(a), y, zc + radius * np.sin(a)], axis=1)

    def radial(a):
        return np.stack([np.cos(a), np.zeros_like(a), np.sin(a)], axis=1)

    corners = [point(a0, y0), point(a1, y0), point(a1, y1), point(a0, y1)]
    rads = [radial(a0), radial(a1), radial(a1), radial(a0)]
    tris, rad = [], []
    for k in ((0, 1, 2), (0, 2, 3)):
        v0, v1, v2 = (corners[m] for m in k)
        n = np.cross(v1 - v0, v2 - v0)
        # orientation: swap the last two corners where the normal points the wrong way
        flip = ((np.sum(n * (rads[k[0]] + rads[k[1]] + rads[k[2]]), axis=1) > 0) != outward)[:, None]
        tris.append(np.concatenate([v0, np.where(flip, v2, v1), np.where(flip, v1, v2)], axis=1))
        rad.append(np.concatenate([rads[k[0]], np.where(flip, rads[k[2]], rads[k[1]]),
                                   np.where(flip, rads[k[1]], rads[k[2]])], axis=1))
    return np.stack(tris, axis=1).reshape(-1, 9), np.stack(rad, axis=1).reshape(-1, 9)


def random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


# --------------------------------------------------------------------------------------------
# descriptors
# --------------------------------------------------------------------------------------------
def acquisition(n_elem, pitch, n_samples, angles_deg, n_rays, k_max, c_bf, fs=40e6, bw=0.6, h_el=5 * MM,
                alpha_m_deg=20.0, alpha_c_deg=45.0, split_mode=0, split_q=0.5, stream_id=0, tx_elem=-1,
                n_tx_elem=0, rough_nee=1):
    return dict(n_elem=int(n_elem), pitch=float(pitch), h_el=float(h_el), fs=float(fs),
                n_samples=int(n_samples), k_max=int(k_max), n_rays=int(n_rays), bw=float(bw),
                alpha_m=alpha_m_deg * DEG, alpha_c=alpha_c_deg * DEG, c_bf=float(c_bf),
                split_mode=int(split_mode), split_q=float(split_q), stream_id=int(stream_id),
                tx_elem=int(tx_elem), n_tx_elem=int(n_tx_elem), rough_nee=int(rough_nee),
                angles=[float(a) * DEG for a in angles_deg])


def image(n_lines, n_depth, x0, x1, z0, z1, dr_db=60.0, lambda1=0.0, lambda2=1.0, f_number=0.0):
    """Image grid; f_number > 0 selects a dynamic receive aperture (0: the whole array)."""
    return dict(n_lines=int(n_lines), n_depth=int(n_depth), x0=float(x0), x1=float(x1), z0=float(z0),
                z1=float(z1), dr_db=float(dr_db), lambda1=float(lambda1), lambda2=float(lambda2),
                f_number=float(f_number))


def theta_vector(media, amp_scale=1.0, f0=5e6):
    """media: list of (c, rho, alpha) -> flat theta."""
    th = []
    for c, r, a in media:
        th += [float(c), float(r), float(a)]
    return np.asarray(th + [float(amp_scale), float(f0)], dtype=np.float64)


def empty_scatterers():
    return np.zeros((0, 3)), np.zeros((0,))


# --------------------------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------------------------
def two_layer(n_rays=10000, k_max=4, n_samples=2048, n_depth=1024, n_lines=128, n_elem=64):
    tris = box_mesh((-20 * MM, -20 * MM, 20 * MM), (20 * MM, 20 * MM, 40 * MM))
    media = np.tile(np.array([[0, 1]], dtype=np.int32), (len(tris), 1))
    sp, sa = empty_scatterers()
    theta = theta_vector([(1480.0, 1000.0, 0.002), (1540.0, 1060.0, 0.5)])
    pitch = 0.3 * MM
    acq = acquisition(n_elem, pitch, n_samples, [0.0], n_rays, k_max, 1480.0)
    fs = acq["fs"]
    zmax = 1480.0 * (n_samples - 1) / (2 * fs)
    half = 0.5 * (n_elem - 1) * pitch
    img = image(n_lines, n_depth, -half, half, 0.0, zmax)
    return dict(name="two_layer", tris=tris, media=media, scat_pos=sp, scat_amp=sa, r_s=0.1 * MM, M=2,
                theta=theta, acq=acq, img=img, seed=0)


def place_ellipsoids(rng, n, box_lo, box_hi, semi_lo, semi_hi, margin=1.0 * MM, max_tries=100000):
    centers, semis, rots = [], [], []
    tries = 0
    while len(centers) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("ellipsoid placement failed")
        semi = rng.uniform(semi_lo, semi_hi, size=3)
        r = semi.max()
        c = np.array([rng.uniform(box_lo[i] + r + margin, box_hi[i] - r - margin) for i in range(3)])
        if any(np.linalg.norm(c - c2) < r + s2.max() + margin for c2, s2 in zip(centers, semis)):
            continue
        centers.append(c)
        semis.append(semi)
        rots.append(random_rotation(rng))
    return centers, semis, rots


def inclusions(n_regions=12, n_scat=100000, n_rays=7813, k_max=8, n_samples=4096, angles_deg=None,
               n_lines=256, n_depth=1024, n_elem=128, n_lat=65, n_lon=130, seed_geom=2, seed_scat=3):
    box_lo = (-20 * MM, -20 * MM, 0.0)
    box_hi = (20 * MM, 20 * MM, 60 * MM)
    rng = np.random.default_rng(seed_geom)
    # keep every region clear of the probe face (z >= 3 mm)
    centers, semis, rots = place_ellipsoids(rng, n_regions, (box_lo[0], box_lo[1], 3 * MM), box_hi,
                                            2 * MM, 6 * MM)
    tris, media = [], []
    for i, (c, s, r) in enumerate(zip(centers, semis, rots)):
        t = ellipsoid_mesh(c, s, r, n_lat=n_lat, n_lon=n_lon)
        tris.append(t)
        media.append(np.tile(np.array([[0, i + 1]], dtype=np.int32), (len(t), 1)))
    tris = np.concatenate(tris) if tris else np.zeros((0, 9))
    media = np.concatenate(media) if media else np.zeros((0, 2), dtype=np.int32)
    mats = [(1540.0, 1000.0, 0.5)]
    for _ in range(n_regions):
        mats.append((rng.uniform(1450, 1650), rng.uniform(950, 1150), rng.uniform(0.3, 1.0)))
    theta = theta_vector(mats)
    rng_s = np.random.default_rng(seed_scat)
    sp = np.stack([rng_s.uniform(box_lo[i], box_hi[i], size=n_scat) for i in range(3)], axis=1)
    sa = rng_s.normal(size=n_scat)
    if angles_deg is None:
        angles_deg = list(np.linspace(-15.0, 15.0, 16))
    pitch = 0.3 * MM
    acq = acquisition(n_elem, pitch, n_samples, angles_deg, n_rays, k_max, 1540.0)
    half = 0.5 * (n_elem - 1) * pitch
    img = image(n_lines, n_depth, -half, half, 0.0, 60 * MM)
    return dict(name="inclusions", tris=tris, media=media, scat_pos=sp, scat_amp=sa, r_s=0.1 * MM,
                M=n_regions + 1, theta=theta, acq=acq, img=img, seed=0)


def differentiation(n_rays=782, **kw):
    w = inclusions(angles_deg=[0.0], k_max=4, n_rays=n_rays, **kw)
    w["name"] = "differentiation"
    w["theta_target"] = perturbed_theta(w["theta"], 7)
    return w


def slab_scatterers(n_rays=2000, n_scat=1000, k_max=4, seed_scat=3):
    w = two_layer(n_rays=n_rays, k_max=k_max)
    rng = np.random.default_rng(seed_scat)
    sp = np.stack([rng.uniform(-18 * MM, 18 * MM, n_scat), rng.uniform(-2 * MM, 2 * MM, n_scat),
                   rng.uniform(21 * MM, 37 * MM, n_scat)], axis=1)
    w.update(name="slab_scatterers", scat_pos=sp, scat_amp=rng.normal(size=n_scat))
    w["theta_target"] = perturbed_theta(w["theta"], 7)
    return w


def hollow_cylinder_mesh(radius=5 * MM, wall=1 * MM, depth=15 * MM, half_len=8 * MM, n_phi=96, n_y=6):
    """The tube's triangles and media and d tris / d radius (both surfaces move outward, the
    wall thickness fixed): outer surface (tissue | wall) with outward normals, inner surface
    (lumen | wall) with normals toward the axis."""
    outer, r_out = tube_mesh(radius, depth, half_len, n_phi, n_y, outward=True)
    inner, r_in = tube_mesh(radius - wall, depth, half_len, n_phi, n_y, outward=False)
    media = np.concatenate([np.tile(np.array([[0, 1]], dtype=np.int32), (len(outer), 1)),
                            np.tile(np.array([[2, 1]], dtype=np.int32), (len(inner), 1))])
    return np.concatenate([outer, inner]), media, np.concatenate([r_out, r_in])


def hollow_cylinder(radius=5 * MM, wall=1 * MM, depth=15 * MM, n_rays=2000, n_scat=3000, k_max=4, n_phi=96,
                    n_y=6, half_len=8 * MM, angles_deg=(0.0,), n_elem=64, n_samples=2048, seed_scat=11):
    """Tube along y at depth `depth` (axis), see hollow_cylinder_mesh.  Media: 0 tissue,
    1 wall, 2 lumen fluid.  Scatterers uniform in the imaged slab outside the lumen."""
    tris, media, dtris_dR = hollow_cylinder_mesh(radius, wall, depth, half_len, n_phi, n_y)
    rng = np.random.default_rng(seed_scat)
    pts = []
    while len(pts) < n_scat:
        p = np.array([rng.uniform(-10 * MM, 10 * MM), rng.uniform(-2 * MM, 2 * MM), rng.uniform(4 * MM, 28 * MM)])
        if math.hypot(p[0], p[2] - depth) > radius - wall + 0.2 * MM:
            pts.append(p)
    sp = np.asarray(pts)
    sa = rng.normal(size=n_scat)
    theta = theta_vector([(1540.0, 1000.0, 0.5), (1600.0, 1100.0, 0.8), (1480.0, 1000.0, 0.002)])
    pitch = 0.3 * MM
    acq = acquisition(n_elem, pitch, n_samples, list(angles_deg), n_rays, k_max, 1540.0)
    half = 0.5 * (n_elem - 1) * pitch
    img = image(128, 512, -half, half, 5 * MM, 30 * MM)
    w = dict(name="hollow_cylinder", tris=tris, media=media, scat_pos=sp, scat_amp=sa, r_s=0.1 * MM, M=3,
             theta=theta, acq=acq, img=img, seed=0, radius=float(radius), dtris_dR=dtris_dR)
    w["theta_target"] = perturbed_theta(theta, 7)
    return w


def with_roughness(w, rough):
    """The workload with rough interfaces: theta (and theta_target) extended by a GGX roughness
    per medium, the roughness of the interfaces bounding that medium (triangles whose back side
    it is)."""
    w = dict(w)
    r = np.asarray(rough, dtype=np.float64)
    assert r.shape == (w["M"],)
    w["rough"] = True
    w["theta"] = np.concatenate([np.asarray(w["theta"], np.float64), r])
    if "theta_target" in w:
        w["theta_target"] = np.concatenate([np.asarray(w["theta_target"], np.float64), r])
    return w


def perturbed_theta(theta, seed, frac=0.05):
    rng = np.random.default_rng(seed)
    s = rng.choice([-1.0, 1.0], size=len(theta))
    return np.asarray(theta) * (1.0 + frac * s)


def rays_for(total_rays_per_tx, n_elem):
    return int(math.ceil(total_rays_per_tx / n_elem))


def batch_workloads(n=256, seed=4, scale=1.0, rng_sizes=None):
    """Scenes of uneven size for batched runs: triangle counts log-uniform in [1e3, 3e5] (1-12
    ellipsoids, tessellation scaled), rays per transmit log-uniform in [1e4, 1e6], 64/128/192
    elements, 1024/2048/4096 samples, 1-16 plane waves over +-15 deg (one: 0 deg), scatterers
    log-uniform in [1e3, 1e5]; even indices forward only, odd forward + adjoint.  `scale`
    multiplies ray and scatterer counts (smaller test batches)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        n_tris = float(np.exp(rng.uniform(np.log(1e3), np.log(3e5))))
        n_reg = int(rng.integers(1, 13))
        per = n_tris / n_reg  # 2 n_lon (n_lat - 1) triangles per ellipsoid, n_lon = 2 n_lat
        n_lat = max(4, int(round((1 + math.sqrt(1 + 4 * per)) / 4)))
        rays_tx = float(np.exp(rng.uniform(np.log(1e4), np.log(1e6)))) * scale
        n_elem = int(rng.choice([64, 128, 192]))
        n_samples = int(rng.choice([1024, 2048, 4096]))
        n_tx = int(rng.integers(1, 17))
        angles = [0.0] if n_tx == 1 else list(np.linspace(-15.0, 15.0, n_tx))
        n_scat = max(10, int(np.exp(rng.uniform(np.log(1e3), np.log(1e5))) * scale))
        w = inclusions(n_regions=n_reg, n_scat=n_scat, n_rays=max(1, int(math.ceil(rays_tx / n_elem))), k_max=8,
                       n_samples=n_samples, angles_deg=angles, n_lines=128, n_depth=512, n_elem=n_elem,
                       n_lat=n_lat, n_lon=2 * n_lat, seed_geom=1000 + i, seed_scat=2000 + i)
        depth = min(60 * MM, 1540.0 * (n_samples - 1) / (2 * w["acq"]["fs"]))
        w["img"] = image(128, 512, w["img"]["x0"], w["img"]["x1"], 0.0, depth)
        w["name"] = "batch-%d" % i
        w["seed"] = i
        w["adjoint"] = bool(i % 2)
        if w["adjoint"]:
            w["theta_target"] = perturbed_theta(w["theta"], 7 + i)
        out.append(w)
    return out
