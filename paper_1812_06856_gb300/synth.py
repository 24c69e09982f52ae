"""Seeded synthetic light-field inputs: camera rigs, ray-cast scenes, grid label maps.

This module is the only code shared by the CUDA path's tests/bench and the
FP64 oracle's tests.  It produces *inputs* (cameras, RGB views, superpixel
label maps, ground truth) and holds none of the depth method's arithmetic:
no plane sweep, no photo-consistency, no energy, no propagation.

Camera convention (the one the C ABI uses): a world point X maps to camera
coordinates x = R X + t; pixel = K x / x_z with pixel centres at integer
coordinates (0..W-1, 0..H-1), x right, y down, z forward.  K is pinhole
(last row 0 0 1).

The scenes stand in for the paper's camera-array datasets (Middlebury
multi-view, Stanford/ULB/Fraunhofer light fields, Section IV): planar
rectangles and spheres with hashed value-noise textures at a 2-4 px feature
scale at the nearest depth, optionally untextured, in front of a far
background plane.  Superpixel label maps are regular (or seeded-perturbed)
grids standing in for SLIC over-segmentation (Section III-A).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

__all__ = [
    "Rig", "PlaneObj", "SphereObj", "Scene", "LightField",
    "line_rig", "grid_rig", "arc_rig", "render", "grid_labels",
    "make_config", "quantize_rgba8", "to_rgba_float", "gt_planes",
    "CONFIG_NAMES",
]


# ----------------------------------------------------------------------------
# Rigs
# ----------------------------------------------------------------------------

@dataclass
class Rig:
    K: np.ndarray  # (V,3,3) float64
    R: np.ndarray  # (V,3,3) float64, world -> camera
    t: np.ndarray  # (V,3)   float64
    W: int
    H: int

    @property
    def V(self) -> int:
        return self.K.shape[0]

    def centres(self) -> np.ndarray:
        return np.einsum("vji,vj->vi", self.R, -self.t)


def _intrinsics(f: float, W: int, H: int) -> np.ndarray:
    return np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])


def _look_at(C: np.ndarray, target: np.ndarray):
    z = target - C
    z = z / np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    x = x / np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ C
    return R, t


def line_rig(V: int, baseline: float, f: float, W: int, H: int) -> Rig:
    """V parallel cameras on the x axis, centred at the origin, looking +z."""
    K = np.stack([_intrinsics(f, W, H)] * V)
    R = np.stack([np.eye(3)] * V)
    xs = (np.arange(V) - (V - 1) / 2.0) * baseline
    t = np.stack([-np.array([x, 0.0, 0.0]) for x in xs])
    return Rig(K, R, t, W, H)


def grid_rig(rows: int, cols: int, baseline: float, f: float, W: int, H: int) -> Rig:
    """rows x cols parallel cameras in the z=0 plane, row-major order."""
    V = rows * cols
    K = np.stack([_intrinsics(f, W, H)] * V)
    R = np.stack([np.eye(3)] * V)
    ts = []
    for r in range(rows):
        for c in range(cols):
            C = np.array([(c - (cols - 1) / 2.0) * baseline, (r - (rows - 1) / 2.0) * baseline, 0.0])
            ts.append(-C)
    return Rig(K, R, np.stack(ts), W, H)


def arc_rig(V: int, arc_deg: float, radius: float, f: float, W: int, H: int) -> Rig:
    """V cameras on a horizontal circular arc of `arc_deg` degrees and the given
    radius around the scene centre (0,0,radius), all facing that centre."""
    centre = np.array([0.0, 0.0, radius])
    K = np.stack([_intrinsics(f, W, H)] * V)
    Rs, ts = [], []
    for v in range(V):
        a = math.radians(arc_deg) * ((v / (V - 1)) - 0.5) if V > 1 else 0.0
        C = centre + radius * np.array([math.sin(a), 0.0, -math.cos(a)])
        R, t = _look_at(C, centre)
        Rs.append(R)
        ts.append(t)
    return Rig(K, np.stack(Rs), np.stack(ts), W, H)


# ----------------------------------------------------------------------------
# Scene objects and rendering
# ----------------------------------------------------------------------------

@dataclass
class PlaneObj:
    centre: np.ndarray
    normal: np.ndarray
    u_axis: np.ndarray
    v_axis: np.ndarray
    half_u: float
    half_v: float
    base: np.ndarray            # RGB base colour in [0,1]
    texture: str = "noise"      # "noise" | "flat" | "affine"
    feat: float = 0.02          # noise feature size in metres
    amp: float = 0.8
    seed: int = 0
    affine: np.ndarray | None = None  # (3,3): colour_c = a[c,0] + a[c,1]*s + a[c,2]*t


@dataclass
class SphereObj:
    centre: np.ndarray
    radius: float
    base: np.ndarray
    texture: str = "noise"
    feat: float = 0.02
    amp: float = 0.8
    seed: int = 0


@dataclass
class Scene:
    planes: list = field(default_factory=list)
    spheres: list = field(default_factory=list)

    def translated(self, delta_per_obj: list) -> "Scene":
        """Copy with object i moved by delta_per_obj[i] (planes first, then spheres)."""
        out = Scene()
        k = 0
        for p in self.planes:
            q = PlaneObj(**{**p.__dict__})
            q.centre = p.centre + delta_per_obj[k]
            out.planes.append(q)
            k += 1
        for s in self.spheres:
            q = SphereObj(**{**s.__dict__})
            q.centre = s.centre + delta_per_obj[k]
            out.spheres.append(q)
            k += 1
        return out


def _hash01(i, j, k, c: int, seed: int):
    """Integer lattice hash -> uniform [0,1) (int64 torch tensors, values < 2^31)."""
    h = (i * 73856093) ^ (j * 19349663) ^ (k * 83492791) ^ ((c * 2654435761 + seed * 40503) % (1 << 31))
    h = h & 0x7FFFFFFF
    for _ in range(3):
        h = ((h * 1103515245 + 12345) & 0x7FFFFFFF) ^ (h >> 13)
    return h.to(torch.float64) / float(1 << 31)


def _smooth(f):
    return f * f * (3.0 - 2.0 * f)


def _value_noise2(s, t, c: int, seed: int):
    i0 = torch.floor(s)
    j0 = torch.floor(t)
    fs = _smooth(s - i0)
    ft = _smooth(t - j0)
    i0 = i0.to(torch.int64)
    j0 = j0.to(torch.int64)
    z = torch.zeros_like(i0)
    n00 = _hash01(i0, j0, z, c, seed)
    n10 = _hash01(i0 + 1, j0, z, c, seed)
    n01 = _hash01(i0, j0 + 1, z, c, seed)
    n11 = _hash01(i0 + 1, j0 + 1, z, c, seed)
    return (n00 * (1 - fs) + n10 * fs) * (1 - ft) + (n01 * (1 - fs) + n11 * fs) * ft


def _value_noise3(x, y, z, c: int, seed: int):
    i0, j0, k0 = torch.floor(x), torch.floor(y), torch.floor(z)
    fx, fy, fz = _smooth(x - i0), _smooth(y - j0), _smooth(z - k0)
    i0, j0, k0 = i0.to(torch.int64), j0.to(torch.int64), k0.to(torch.int64)
    out = torch.zeros_like(x)
    for di in (0, 1):
        wx = fx if di else 1 - fx
        for dj in (0, 1):
            wy = fy if dj else 1 - fy
            for dk in (0, 1):
                wz = fz if dk else 1 - fz
                out = out + wx * wy * wz * _hash01(i0 + di, j0 + dj, k0 + dk, c, seed)
    return out


def _noise_colour(coords, base, amp, seed):
    cols = []
    for c in range(3):
        if len(coords) == 2:
            n = _value_noise2(coords[0], coords[1], c, seed) + 0.5 * _value_noise2(
                2 * coords[0] + 17.0, 2 * coords[1] + 31.0, c, seed + 7)
        else:
            n = _value_noise3(*coords, c, seed) + 0.5 * _value_noise3(
                2 * coords[0] + 17.0, 2 * coords[1] + 31.0, 2 * coords[2] + 5.0, c, seed + 7)
        n = n / 1.5
        cols.append(torch.clamp(base[c] + amp * (n - 0.5), 0.0, 1.0))
    return torch.stack(cols, dim=-1)


def render(rig: Rig, scene: Scene, device="cpu"):
    """Ray-cast every view at pixel centres.

    Returns (rgb (V,H,W,3) float64 in [0,1], depth (V,H,W) camera z, obj (V,H,W)
    int32 object index: planes 0..P-1, spheres P.., -1 = miss)."""
    dev = torch.device(device)
    V, W, H = rig.V, rig.W, rig.H
    vv, uu = torch.meshgrid(torch.arange(H, dtype=torch.float64, device=dev),
                            torch.arange(W, dtype=torch.float64, device=dev), indexing="ij")
    ones = torch.ones_like(uu)
    pix = torch.stack([uu, vv, ones], dim=-1)  # (H,W,3)
    rgb_all, dep_all, obj_all = [], [], []
    for v in range(V):
        Kinv = torch.tensor(np.linalg.inv(rig.K[v]), device=dev)
        R = torch.tensor(rig.R[v], device=dev)
        t = torch.tensor(rig.t[v], device=dev)
        dc = pix @ Kinv.T                    # camera-frame ray, z = 1
        dw = dc @ R                          # world direction (R^T dc)
        C = -(R.T @ t)                       # camera centre
        best = torch.full((H, W), float("inf"), dtype=torch.float64, device=dev)
        obj = torch.full((H, W), -1, dtype=torch.int32, device=dev)
        rgb = torch.zeros((H, W, 3), dtype=torch.float64, device=dev)
        k = 0
        for p in scene.planes:
            N = torch.tensor(p.normal, device=dev)
            P0 = torch.tensor(p.centre, device=dev)
            denom = dw @ N
            lam = ((P0 - C) @ N) / torch.where(denom.abs() < 1e-15, torch.full_like(denom, 1e-15), denom)
            X = C + lam[..., None] * dw
            rel = X - P0
            s = rel @ torch.tensor(p.u_axis, device=dev)
            tt = rel @ torch.tensor(p.v_axis, device=dev)
            hit = (lam > 1e-9) & (s.abs() <= p.half_u) & (tt.abs() <= p.half_v) & (lam < best)
            if hit.any():
                base = torch.tensor(p.base, device=dev)
                if p.texture == "noise":
                    col = _noise_colour((s / p.feat, tt / p.feat), base, p.amp, p.seed)
                elif p.texture == "affine":
                    a = torch.tensor(p.affine, device=dev)
                    col = a[:, 0] + s[..., None] * a[:, 1] + tt[..., None] * a[:, 2]
                else:
                    col = base.expand(H, W, 3)
                rgb = torch.where(hit[..., None], col, rgb)
                best = torch.where(hit, lam, best)
                obj = torch.where(hit, torch.full_like(obj, k), obj)
            k += 1
        for sp in scene.spheres:
            S = torch.tensor(sp.centre, device=dev)
            oc = C - S
            a = (dw * dw).sum(-1)
            b = 2.0 * (dw @ oc)
            c = float(oc @ oc) - sp.radius ** 2
            disc = b * b - 4 * a * c
            sq = torch.sqrt(torch.clamp(disc, min=0.0))
            lam = (-b - sq) / (2 * a)
            hit = (disc > 0) & (lam > 1e-9) & (lam < best)
            if hit.any():
                X = C + lam[..., None] * dw - S
                base = torch.tensor(sp.base, device=dev)
                if sp.texture == "noise":
                    col = _noise_colour((X[..., 0] / sp.feat, X[..., 1] / sp.feat, X[..., 2] / sp.feat),
                                        base, sp.amp, sp.seed)
                else:
                    col = base.expand(H, W, 3)
                rgb = torch.where(hit[..., None], col, rgb)
                best = torch.where(hit, lam, best)
                obj = torch.where(hit, torch.full_like(obj, k), obj)
            k += 1
        # camera-frame ray has z = 1, so the ray parameter is the depth
        depth = torch.where(torch.isfinite(best), best, torch.zeros_like(best))
        rgb_all.append(rgb)
        dep_all.append(depth)
        obj_all.append(obj)
    return torch.stack(rgb_all), torch.stack(dep_all), torch.stack(obj_all)


def quantize_rgba8(rgb: torch.Tensor) -> torch.Tensor:
    """(...,3) float in [0,1] -> (...,4) uint8 RGBA (alpha 255)."""
    q = torch.clamp(torch.floor(rgb * 255.0 + 0.5), 0, 255).to(torch.uint8)
    a = torch.full(q.shape[:-1] + (1,), 255, dtype=torch.uint8, device=q.device)
    return torch.cat([q, a], dim=-1).contiguous()


def to_rgba_float(rgb: torch.Tensor, dtype=torch.float32) -> torch.Tensor:
    a = torch.ones(rgb.shape[:-1] + (1,), dtype=rgb.dtype, device=rgb.device)
    return torch.cat([rgb, a], dim=-1).to(dtype).contiguous()


# ----------------------------------------------------------------------------
# Superpixel label maps (stand-in for SLIC, Section III-A)
# ----------------------------------------------------------------------------

def _rnd(x: float) -> int:
    return int(math.floor(x + 0.5))


def grid_labels(W: int, H: int, pitch: float, perturb: bool = False, seed: int = 0):
    """Regular grid label map with GW = round(W/pitch), GH = round(H/pitch),
    cell boundaries at round(k*W/GW); label = gy*GW + gx.  With `perturb`,
    each interior boundary is shifted per row/column segment by a seeded
    uniform integer in [-floor(pitch/4), floor(pitch/4)]."""
    GW = max(1, _rnd(W / pitch))
    GH = max(1, _rnd(H / pitch))
    bx = np.array([_rnd(k * W / GW) for k in range(GW + 1)], dtype=np.int64)
    by = np.array([_rnd(k * H / GH) for k in range(GH + 1)], dtype=np.int64)
    u = np.arange(W)
    v = np.arange(H)
    if not perturb:
        gx = np.searchsorted(bx, u, side="right") - 1
        gy = np.searchsorted(by, v, side="right") - 1
        lab = gy[:, None] * GW + gx[None, :]
        return lab.astype(np.int32), GW, GH
    rng = np.random.default_rng(seed)
    m = int(math.floor(pitch / 4))
    sx = rng.integers(-m, m + 1, size=(GH, GW + 1))
    sy = rng.integers(-m, m + 1, size=(GW, GH + 1))
    sx[:, 0] = 0
    sx[:, GW] = 0
    sy[:, 0] = 0
    sy[:, GH] = 0
    gx0 = np.searchsorted(bx, u, side="right") - 1                     # unperturbed column per u
    byp = by[None, :] + sy                                             # (GW, GH+1) per column cell
    gy = np.empty((H, W), dtype=np.int64)
    for c in range(GW):
        cols = np.nonzero(gx0 == c)[0]
        gyc = np.searchsorted(byp[c], v, side="right") - 1
        gy[:, cols] = np.clip(gyc, 0, GH - 1)[:, None]
    bxp = bx[None, :] + sx                                             # (GH, GW+1) per row cell
    gx = np.empty((H, W), dtype=np.int64)
    for r in range(GH):
        rows_r = gy == r
        gxr = np.clip(np.searchsorted(bxp[r], u, side="right") - 1, 0, GW - 1)
        gx[rows_r] = np.broadcast_to(gxr[None, :], (H, W))[rows_r]
    lab = gy * GW + gx
    return lab.astype(np.int32), GW, GH


# ----------------------------------------------------------------------------
# Workload configurations (shapes of the paper's workloads, Table I / Sec. IV)
# ----------------------------------------------------------------------------

@dataclass
class LightField:
    name: str
    rig: Rig
    scene: Scene
    rgb: torch.Tensor       # (V,H,W,3) float64
    depth: torch.Tensor     # (V,H,W) ground-truth camera z
    obj: torch.Tensor       # (V,H,W) object id
    labels: np.ndarray      # (V,H,W) int32
    GW: int
    GH: int
    params: dict
    pitch: float


CONFIG_NAMES = {
    1: "plain-3x320x240",
    2: "plain-8x1024x768-arc",
    3: "precision-16x1920x1080-grid",
}

SCENE_SEED_BASE = 1812068560


def _rand_unit_colour(rng):
    return rng.uniform(0.15, 0.85, size=3)


def _slanted_plane(rng, centre, tilt_deg, axis, half_u, half_v, feat, textured=True, seed=0):
    """A rectangle facing the cameras (-z), tilted by tilt_deg about `axis` ('x' or 'y')."""
    a = math.radians(tilt_deg)
    if axis == "y":
        n = np.array([math.sin(a), 0.0, -math.cos(a)])
        ua = np.array([math.cos(a), 0.0, math.sin(a)])
        va = np.array([0.0, 1.0, 0.0])
    else:
        n = np.array([0.0, math.sin(a), -math.cos(a)])
        ua = np.array([1.0, 0.0, 0.0])
        va = np.array([0.0, math.cos(a), math.sin(a)])
    return PlaneObj(np.asarray(centre, float), n, ua, va, half_u, half_v, _rand_unit_colour(rng),
                    "noise" if textured else "flat", feat, 0.8, seed)


def _scene_config1(rng, f, W, H, d_min, d_max):
    feat = 3.0 * d_min / f
    sc = Scene()
    seed = int(rng.integers(1 << 20))
    # background (fronto-parallel, fills the view)
    sc.planes.append(_slanted_plane(rng, [0, 0, 4.6], 0.0, "y", 50.0, 50.0, feat * 2.0, True, seed + 1))
    # fronto-parallel rectangle
    sc.planes.append(_slanted_plane(rng, [-0.35, -0.1, 2.2], 0.0, "y", 0.35, 0.3, feat, True, seed + 2))
    # slanted planes (<= 40 degrees)
    sc.planes.append(_slanted_plane(rng, [0.45, 0.05, 3.2], 35.0, "y", 0.45, 0.5, feat, True, seed + 3))
    sc.planes.append(_slanted_plane(rng, [-0.1, 0.55, 1.8], 30.0, "x", 0.5, 0.18, feat, True, seed + 4))
    return sc


def _random_scene(rng, n_planes, n_untextured, n_spheres, f, d_min, d_max, spread):
    feat = 3.0 * d_min / f
    sc = Scene()
    seed = int(rng.integers(1 << 20))
    sc.planes.append(_slanted_plane(rng, [0, 0, d_max - 0.4], 0.0, "y", 200.0, 200.0, feat * 2.5, True, seed))
    for k in range(n_planes + n_untextured):
        z = rng.uniform(d_min + 0.6, d_max - 1.2)
        x = rng.uniform(-spread, spread) * z / d_max
        y = rng.uniform(-spread * 0.6, spread * 0.6) * z / d_max
        tilt = rng.uniform(-40.0, 40.0) if rng.uniform() < 0.6 else 0.0
        axis = "x" if rng.uniform() < 0.5 else "y"
        hu = rng.uniform(0.15, 0.5) * z / 4.0
        hv = rng.uniform(0.15, 0.5) * z / 4.0
        textured = k < n_planes
        sc.planes.append(_slanted_plane(rng, [x, y, z], tilt, axis, hu, hv, feat, textured, seed + 11 * (k + 1)))
    for k in range(n_spheres):
        z = rng.uniform(d_min + 0.8, d_max - 1.5)
        x = rng.uniform(-spread, spread) * z / d_max
        y = rng.uniform(-spread * 0.6, spread * 0.6) * z / d_max
        r = rng.uniform(0.12, 0.3) * z / 4.0
        sc.spheres.append(SphereObj(np.array([x, y, z]), r, _rand_unit_colour(rng), "noise", feat, 0.8,
                                    seed + 1000 + 13 * k))
    return sc


def make_config(idx: int, device="cpu", scale: float = 1.0, views: int | None = None) -> LightField:
    """Build config `idx` (1: 3x320x240 line rig, 2: 8x1024x768 arc, 3: 16x1920x1080
    4x4 grid).  `scale` < 1 shrinks the resolution (tests); `views` overrides V."""
    rng = np.random.default_rng(SCENE_SEED_BASE + idx)
    if idx == 1:
        W, H = _rnd(320 * scale), _rnd(240 * scale)
        f = 300.0 * W / 320.0
        V = views or 3
        rig = line_rig(V, 0.1, f, W, H)
        d_min, d_max = 1.0, 5.0
        scene = _scene_config1(rng, f, W, H, d_min, d_max)
        pitch, perturb = 16.0 * scale if scale < 1 else 16.0, False
        params = dict(d_min=d_min, d_max=d_max, num_labels=64, iterations=4)
    elif idx == 2:
        W, H = _rnd(1024 * scale), _rnd(768 * scale)
        f = 300.0 * W / 320.0
        V = views or 8
        rig = arc_rig(V, 30.0, 5.0, f, W, H)
        d_min, d_max = 2.0, 8.0
        scene = _random_scene(rng, 12, 3, 4, f, d_min, d_max, 1.6)
        pitch, perturb = 14.0, True
        params = dict(d_min=d_min, d_max=d_max, num_labels=256, iterations=6)
    elif idx == 3:
        W, H = _rnd(1920 * scale), _rnd(1080 * scale)
        f = 300.0 * W / 320.0
        V = views or 16
        rows = int(round(math.sqrt(V)))
        cols = V // rows
        rig = grid_rig(rows, cols, 0.08, f, W, H)
        d_min, d_max = 2.0, 8.0
        n_planes = 30
        scene = _random_scene(rng, n_planes - 6, 6, 10, f, d_min, d_max, 2.2)
        pitch, perturb = 16.0, False
        params = dict(d_min=d_min, d_max=d_max, num_labels=256, iterations=8)
    else:
        raise ValueError(f"unknown config {idx}")
    rgb, depth, obj = render(rig, scene, device)
    labs = []
    GW = GH = None
    for v in range(rig.V):
        lab, GW, GH = grid_labels(W, H, pitch, perturb, seed=SCENE_SEED_BASE + 100 * idx + v)
        labs.append(lab)
    return LightField(CONFIG_NAMES[idx] if scale == 1 and views is None else f"{CONFIG_NAMES[idx]}@{scale}",
                      rig, scene, rgb, depth, obj, np.stack(labs), GW, GH, params, pitch)


def gt_planes(lf: LightField) -> np.ndarray:
    """Per (view, SP) ground-truth plane {d, nx, ny, nz} (camera frame, anchored
    at the SP centroid) of the planar object covering most of the SP; rows of
    zeros where the majority object is a sphere or missing.  Returns (V, S, 4)."""
    rig = lf.rig
    S = lf.GW * lf.GH
    out = np.zeros((rig.V, S, 4))
    n_planes = len(lf.scene.planes)
    for v in range(rig.V):
        lab = lf.labels[v].reshape(-1)
        obj = lf.obj[v].reshape(-1).cpu().numpy()
        H, W = lf.labels[v].shape
        uu = np.tile(np.arange(W), H).astype(np.float64)
        vv = np.repeat(np.arange(H), W).astype(np.float64)
        cnt = np.bincount(lab, minlength=S).astype(np.float64)
        cu = np.bincount(lab, weights=uu, minlength=S) / np.maximum(cnt, 1)
        cv = np.bincount(lab, weights=vv, minlength=S) / np.maximum(cnt, 1)
        Kinv = np.linalg.inv(rig.K[v])
        R, t = rig.R[v], rig.t[v]
        for s in range(S):
            if cnt[s] == 0:
                continue
            ids = obj[lab == s]
            ids = ids[ids >= 0]
            if ids.size == 0:
                continue
            k = np.bincount(ids).argmax()
            if k >= n_planes:
                continue
            p = lf.scene.planes[k]
            n_c = R @ p.normal                       # camera-frame normal
            X0 = R @ p.centre + t                    # a point of the plane, camera frame
            ray = Kinv @ np.array([cu[s], cv[s], 1.0])
            lam = (n_c @ X0) / (n_c @ ray)
            if n_c @ X0 > 0:
                n_c = -n_c
            out[v, s] = [lam * ray[2], *n_c]
    return out


def method_params(lf: LightField, **over) -> dict:
    """Parameter set for a light field: the configuration's depth range, label
    count and iteration count, plus the defaults of the readings (T = 0.04 on
    RGB in [0,1], sigma = 0 -> 2 x inverse-depth bin width, alpha = 0.1,
    eta = 0.5 (Eq. 11), kernel size = smallest image dimension, kernel step 5
    superpixels (Section IV-A), 8 nearest neighbour views, inverse-depth
    domain, jitter on with seed = scene seed xor 0x5EED)."""
    p = dict(
        d_min=lf.params["d_min"], d_max=lf.params["d_max"],
        num_labels=lf.params["num_labels"], iterations=lf.params["iterations"],
        T=0.04, sigma=0.0, alpha=0.1, eta=0.5,
        kernel_size_init=0, kernel_step_sp=5.0, max_neighbor_views=8,
        depth_domain=0, jitter=1, term_mask=7, sweep_frame=0,
        seed=(SCENE_SEED_BASE ^ 0x5EED), lf_index=0, xy_eps=0.0, warm_iter_offset=0,
        perturb_samples=0, perturb_scale=0.05,
    )
    p.update(over)
    return p


def oracle_inputs(lf: LightField, rgb=None):
    """(K, R, t, rgb list, labels list, GW, GH) as plain numpy arrays.  `rgb`
    overrides the views (e.g. the RGBA8-quantised colours actually given to
    the GPU path, as float64 in [0,1])."""
    r = lf.rgb if rgb is None else rgb
    r = r.detach().cpu().numpy() if isinstance(r, torch.Tensor) else np.asarray(r)
    return (lf.rig.K, lf.rig.R, lf.rig.t, [r[v] for v in range(lf.rig.V)],
            [lf.labels[v] for v in range(lf.rig.V)], lf.GW, lf.GH)


def rgba8_as_float(rgba8: torch.Tensor) -> torch.Tensor:
    """RGBA8 views -> RGB float64 in [0,1] (value / 255)."""
    return rgba8[..., :3].to(torch.float64) / 255.0


# ----------------------------------------------------------------------------
# Serving workload: three rigs filming a scene while moving
# ----------------------------------------------------------------------------

SERVING_RIGS = ("A", "B", "C")


@dataclass
class ServingRig:
    """One rig of the serving workload: `keyframes` rendered frames of the rig
    translated by `step` metres per frame along world x; frame f of the stream
    shows keyframe `keyframe_of(f)` (a ping-pong walk, so consecutive frames
    are always one step apart)."""
    name: str
    rigs: list              # Rig per keyframe
    views: list             # (V,H,W,4) uint8 tensor per keyframe
    labels: torch.Tensor    # (V,H,W) int32, static grid
    GW: int
    GH: int
    params: dict
    step: float

    @property
    def V(self) -> int:
        return self.rigs[0].V

    def keyframe_of(self, f: int) -> int:
        n = len(self.rigs)
        if n == 1:
            return 0
        m = f % (2 * n - 2)
        return m if m < n else 2 * n - 2 - m


def _translated(rig: Rig, d: np.ndarray) -> Rig:
    # the camera centres move by d: t' = t - R d
    t = rig.t - np.einsum("vij,j->vi", rig.R, d)
    return Rig(rig.K.copy(), rig.R.copy(), t, rig.W, rig.H)


def make_serving_rig(name: str, device="cpu", keyframes: int = 4, scale: float = 1.0,
                     step: float = 0.015) -> ServingRig:
    """Rig A: 8 x 1024x768 on a 30-degree arc (superpixel pitch 14, perturbed);
    B: 9 x 1280x720 3x3 grid, baseline 0.08 (pitch 16); C: 16 x 1920x1080 4x4
    grid, baseline 0.08 (pitch 16).  Depth range [2, 8], 256 labels, 6 cold
    iterations; each rig films its own seeded scene while translating `step`
    (<= 2 cm) per frame."""
    idx = {"A": 51, "B": 52, "C": 53}[name]
    rng = np.random.default_rng(SCENE_SEED_BASE + idx)
    if name == "A":
        W, H = _rnd(1024 * scale), _rnd(768 * scale)
        f = 300.0 * W / 320.0
        rig0 = arc_rig(8, 30.0, 5.0, f, W, H)
        pitch, perturb = 14.0, True
        scene = _random_scene(rng, 12, 3, 4, f, 2.0, 8.0, 1.6)
    elif name == "B":
        W, H = _rnd(1280 * scale), _rnd(720 * scale)
        f = 300.0 * W / 320.0
        rig0 = grid_rig(3, 3, 0.08, f, W, H)
        pitch, perturb = 16.0, False
        scene = _random_scene(rng, 16, 4, 6, f, 2.0, 8.0, 2.0)
    elif name == "C":
        W, H = _rnd(1920 * scale), _rnd(1080 * scale)
        f = 300.0 * W / 320.0
        rig0 = grid_rig(4, 4, 0.08, f, W, H)
        pitch, perturb = 16.0, False
        scene = _random_scene(rng, 24, 6, 10, f, 2.0, 8.0, 2.2)
    else:
        raise ValueError(f"unknown serving rig {name}")
    rigs, views = [], []
    for k in range(keyframes):
        rig = _translated(rig0, np.array([step * k, 0.0, 0.0]))
        rgb, _, _ = render(rig, scene, device)
        views.append(quantize_rgba8(rgb))
        rigs.append(rig)
        del rgb
    labs = []
    GW = GH = None
    for v in range(rig0.V):
        lab, GW, GH = grid_labels(W, H, pitch, perturb, seed=SCENE_SEED_BASE + 100 * idx + v)
        labs.append(lab)
    labels = torch.from_numpy(np.ascontiguousarray(np.stack(labs))).to(device)
    params = dict(d_min=2.0, d_max=8.0, num_labels=256, iterations=6,
                  T=0.04, sigma=0.0, alpha=0.1, eta=0.5, kernel_size_init=0, kernel_step_sp=5.0,
                  max_neighbor_views=8, depth_domain=0, jitter=1, term_mask=7, sweep_frame=0,
                  seed=(SCENE_SEED_BASE + idx) ^ 0x5EED, lf_index=0, xy_eps=0.0, warm_iter_offset=0)
    return ServingRig(name, rigs, views, labels, GW, GH, params, step)


# ----------------------------------------------------------------------------
# Batched workload: many independent light fields of uneven shapes
# ----------------------------------------------------------------------------

MIX_RESOLUTIONS = ((640, 480), (1024, 768), (1280, 720), (1920, 1080))


def grid_labels_fast(W: int, H: int, pitch: float, perturb: bool = False, seed: int = 0, device="cpu"):
    """grid_labels computed with batched torch.searchsorted (same RNG draws, same
    result); returns a (H, W) int32 tensor on `device`, GW, GH."""
    GW = max(1, _rnd(W / pitch))
    GH = max(1, _rnd(H / pitch))
    bx = torch.tensor([_rnd(k * W / GW) for k in range(GW + 1)], dtype=torch.int64, device=device)
    by = torch.tensor([_rnd(k * H / GH) for k in range(GH + 1)], dtype=torch.int64, device=device)
    u = torch.arange(W, dtype=torch.int64, device=device)
    v = torch.arange(H, dtype=torch.int64, device=device)
    gx0 = torch.searchsorted(bx, u, right=True) - 1
    if not perturb:
        gy0 = torch.searchsorted(by, v, right=True) - 1
        return (gy0[:, None] * GW + gx0[None, :]).to(torch.int32), GW, GH
    rng = np.random.default_rng(seed)
    m = int(math.floor(pitch / 4))
    sx = rng.integers(-m, m + 1, size=(GH, GW + 1))
    sy = rng.integers(-m, m + 1, size=(GW, GH + 1))
    sx[:, 0] = 0
    sx[:, GW] = 0
    sy[:, 0] = 0
    sy[:, GH] = 0
    byp = by[None, :] + torch.from_numpy(sy).to(device)                # (GW, GH+1) per column cell
    gyc = (torch.searchsorted(byp, v[None, :].expand(GW, H).contiguous(), right=True) - 1).clamp_(0, GH - 1)
    gy = gyc[gx0][:, :].T                                               # (H, W): gyc[gx0[u], v]
    bxp = bx[None, :] + torch.from_numpy(sx).to(device)                # (GH, GW+1) per row cell
    gxr = (torch.searchsorted(bxp, u[None, :].expand(GH, W).contiguous(), right=True) - 1).clamp_(0, GW - 1)
    gx = torch.gather(gxr, 0, gy)                                       # gxr[gy[v,u], u]
    return (gy * GW + gx).to(torch.int32).contiguous(), GW, GH


@dataclass
class MixItem:
    """One light field of the batched workload (views RGBA8 and labels on the device)."""
    rig: Rig
    views: torch.Tensor
    labels: torch.Tensor
    GW: int
    GH: int
    params: dict
    pitch: int
    kind: str

    def item(self) -> dict:
        return dict(views=self.views, labels=self.labels, K=self.rig.K, R=self.rig.R, t=self.rig.t, GW=self.GW,
                    GH=self.GH, params=self.params)


def _mix_shape(rng, scale):
    V = int(rng.integers(4, 17))
    W0, H0 = MIX_RESOLUTIONS[int(rng.integers(len(MIX_RESOLUTIONS)))]
    kind = "arc" if rng.uniform() < 0.5 else "grid"
    pitch = int(rng.integers(8, 33))
    L = int(rng.integers(128, 257))
    return V, _rnd(W0 * scale), _rnd(H0 * scale), kind, pitch, L


def mix_shapes(n: int = 64, scale: float = 1.0, seed: int = SCENE_SEED_BASE + 4) -> list:
    """(views, W, H, rig kind, pitch, labels) of each light field of make_mix, without rendering."""
    return [_mix_shape(np.random.default_rng(seed * 1000 + i), scale) for i in range(n)]


def make_mix(n: int = 64, device="cpu", scale: float = 1.0, seed: int = SCENE_SEED_BASE + 4, first: int = 0) -> list:
    """The batched workload: n independent light fields, camera counts uniform in
    4..16, resolutions from MIX_RESOLUTIONS, arc or grid rigs, perturbed grid
    superpixels of pitch 8..32 px, 128..256 labels, 6 iterations; each with its
    own seeded scene of the config-2 kind and its own jitter key.  `first`
    skips the leading light fields (a sample of the same workload)."""
    out = []
    for i in range(first, n):
        rng = np.random.default_rng(seed * 1000 + i)
        V, W, H, kind, pitch, L = _mix_shape(rng, scale)
        f = 300.0 * W / 320.0
        if kind == "arc":
            rig = arc_rig(V, 30.0, 5.0, f, W, H)
        else:
            rows = max(1, int(math.floor(math.sqrt(V))))
            cols = -(-V // rows)
            g = grid_rig(rows, cols, 0.08, f, W, H)
            rig = Rig(g.K[:V].copy(), g.R[:V].copy(), g.t[:V].copy(), W, H)
        scene = _random_scene(rng, 12, 3, 4, f, 2.0, 8.0, 1.6)
        rgb, _, _ = render(rig, scene, device)
        views = quantize_rgba8(rgb)
        del rgb
        labs, GW, GH = [], None, None
        for v in range(V):
            lab, GW, GH = grid_labels_fast(W, H, pitch * scale if scale < 1 else pitch, True,
                                           seed=seed * 1000 + 100 * i + v, device=device)
            labs.append(lab)
        params = dict(d_min=2.0, d_max=8.0, num_labels=L, iterations=6, T=0.04, sigma=0.0, alpha=0.1, eta=0.5,
                      kernel_size_init=0, kernel_step_sp=5.0, max_neighbor_views=8, depth_domain=0, jitter=1,
                      term_mask=7, sweep_frame=0, seed=(seed * 1000 + i) ^ 0x5EED, lf_index=i, xy_eps=0.0,
                      warm_iter_offset=0)
        out.append(MixItem(rig, views, torch.stack(labs), GW, GH, params, pitch, kind))
    return out
