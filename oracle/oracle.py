"""ctypes wrapper of the FP64 CPU oracle (oracle/lfd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py.  The product package never imports
this module.  Argument marshalling only; all arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfd_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "lfd_fusion_oracle.c"), os.path.join(_HERE, "lfd_slic_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None
REF_MAX = 32          # refinement candidates per superpixel: 8 triangles + up to 24 perturbation samples

MAXN = 8


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (portable flags only)."""
    with _lock:
        stale = not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(f) for f in _SRCS)
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, *_SRCS, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Input(C.Structure):
    _fields_ = [
        ("V", C.c_int32),
        ("W", C.c_void_p), ("H", C.c_void_p), ("GW", C.c_void_p), ("GH", C.c_void_p),
        ("K", C.c_void_p), ("R", C.c_void_p), ("t", C.c_void_p),
        ("rgb", C.c_void_p), ("labels", C.c_void_p),
        ("d_min", C.c_double), ("d_max", C.c_double),
        ("L", C.c_int32),
        ("T", C.c_double), ("sigma", C.c_double), ("alpha", C.c_double), ("eta", C.c_double),
        ("kernel_size_init", C.c_int32),
        ("kernel_step_sp", C.c_double),
        ("max_neighbor_views", C.c_int32),
        ("depth_domain", C.c_int32),
        ("jitter", C.c_int32),
        ("term_mask", C.c_int32),
        ("sweep_frame", C.c_int32),
        ("seed", C.c_uint64),
        ("lf_index", C.c_int32),
        ("xy_eps", C.c_double),
        ("warm_iter_offset", C.c_int32),
        ("perturb_samples", C.c_int32),
        ("perturb_scale", C.c_double),
        ("threads", C.c_int32),
        ("margin_px", C.c_double), ("margin_rel", C.c_double),
    ]


class Terms(C.Structure):
    _fields_ = [
        ("E", C.c_double), ("Es", C.c_double), ("Ec", C.c_double), ("tssd", C.c_double),
        ("E_lo", C.c_double), ("E_hi", C.c_double), ("Ec_lo", C.c_double), ("Ec_hi", C.c_double),
        ("tssd_lo", C.c_double), ("tssd_hi", C.c_double),
        ("S", C.c_double * MAXN), ("Vt", C.c_double * MAXN), ("O", C.c_double * MAXN),
        ("S_lo", C.c_double * MAXN), ("S_hi", C.c_double * MAXN),
        ("V_lo", C.c_double * MAXN), ("V_hi", C.c_double * MAXN),
        ("O_lo", C.c_double * MAXN), ("O_hi", C.c_double * MAXN),
        ("nvalid", C.c_int32 * MAXN), ("nx", C.c_int32 * MAXN), ("ny", C.c_int32 * MAXN),
        ("nflag", C.c_int32 * MAXN),
        ("nviews", C.c_int32),
        ("flag_tssd", C.c_int32), ("flag_energy", C.c_int32),
    ]


class Query(C.Structure):
    _fields_ = [("view", C.c_int32), ("sp", C.c_int32),
                ("d", C.c_double), ("nx", C.c_double), ("ny", C.c_double), ("nz", C.c_double)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp, i32, f64 = C.c_void_p, C.c_int32, C.c_double
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.POINTER(_Input)]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_num_sp.restype = i32
        lib.orc_num_sp.argtypes = [vp, i32]
        lib.orc_sp_base.restype = i32
        lib.orc_sp_base.argtypes = [vp, i32]
        lib.orc_sigma.restype = f64
        lib.orc_sigma.argtypes = [vp]
        lib.orc_delta.restype = f64
        lib.orc_delta.argtypes = [vp]
        lib.orc_sp_stats.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        lib.orc_neighbor_views.restype = i32
        lib.orc_neighbor_views.argtypes = [vp, i32, vp]
        lib.orc_kernel_params.argtypes = [vp, i32, vp, vp]
        lib.orc_kernel_offsets.restype = i32
        lib.orc_kernel_offsets.argtypes = [i32, i32, i32, vp, i32]
        lib.orc_splitmix64.restype = C.c_uint64
        lib.orc_splitmix64.argtypes = [C.c_uint64]
        lib.orc_jitter_u.restype = f64
        lib.orc_jitter_u.argtypes = [C.c_uint64, i32, i32, i32, i32]
        lib.orc_plane_depth.restype = f64
        lib.orc_plane_depth.argtypes = [vp, i32] + [f64] * 8
        lib.orc_project_pixel.restype = i32
        lib.orc_project_pixel.argtypes = [vp, i32, i32] + [f64] * 8 + [vp]
        lib.orc_bilinear_image.argtypes = [vp, i32, i32, f64, f64, vp]
        lib.orc_rasterize.argtypes = [vp, vp, vp, vp]
        lib.orc_sweep.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp]
        lib.orc_iterate.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp, vp, vp, i32, vp]
        lib.orc_refine_candidates.restype = i32
        lib.orc_refine_candidates.argtypes = [vp, vp, i32, f64, f64, f64, f64, i32, vp]
        lib.orc_score.argtypes = [vp, vp, vp, i32, vp]
        lib.orc_fuse.argtypes = [i32, vp, vp, vp, vp, vp, vp, f64, vp, vp]
        lib.orc_rgb_to_lab.argtypes = [vp, vp]
        lib.orc_slic_seeds.argtypes = [i32, i32, vp, i32, i32, vp]
        lib.orc_slic_assign.argtypes = [i32, i32, vp, i32, i32, vp, f64, vp, vp]
        lib.orc_slic_update.argtypes = [i32, i32, vp, i32, i32, vp, vp, vp]
        lib.orc_slic.argtypes = [i32, i32, vp, i32, i32, f64, i32, vp, vp]
        lib.orc_terms_size.restype = i32
        lib.orc_query_size.restype = i32
        lib.orc_input_size.restype = i32
        assert lib.orc_terms_size() == C.sizeof(Terms)
        assert lib.orc_query_size() == C.sizeof(Query)
        assert lib.orc_input_size() == C.sizeof(_Input)
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def jitter_u(seed: int, lf: int, v: int, s: int, k: int) -> float:
    return float(_load().orc_jitter_u(C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), lf, v, s, k))


def kernel_offsets(size_init: int, steps_init: int, it: int) -> np.ndarray:
    lib = _load()
    n = lib.orc_kernel_offsets(size_init, steps_init, it, None, 0)
    out = np.zeros(2 * n, dtype=np.int32)
    lib.orc_kernel_offsets(size_init, steps_init, it, _p(out), n)
    return out.reshape(n, 2)


def bilinear_image(rgb: np.ndarray, x: float, y: float) -> np.ndarray:
    rgb = np.ascontiguousarray(rgb, dtype=np.float64)
    out = np.zeros(3)
    _load().orc_bilinear_image(_p(rgb), rgb.shape[1], rgb.shape[0], x, y, _p(out))
    return out


def fuse(K, R, t, depths, tau: float = 0.01):
    """Stability-based depth fusion (Section III-D), lfd_fusion_oracle.c.
    K, R, t: (V,3,3), (V,3,3), (V,3); depths: list of (H_v, W_v) arrays.
    Returns (fused depths, flags) as lists of arrays."""
    lib = _load()
    V = len(depths)
    K = np.ascontiguousarray(K, dtype=np.float64).reshape(V, 9)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(V, 9)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(V, 3)
    ds = [np.ascontiguousarray(d, dtype=np.float64) for d in depths]
    W = np.array([d.shape[1] for d in ds], dtype=np.int32)
    H = np.array([d.shape[0] for d in ds], dtype=np.int32)
    outs = [np.zeros_like(d) for d in ds]
    flags = [np.zeros(d.shape, dtype=np.uint8) for d in ds]
    arr = lambda xs: (C.c_void_p * V)(*[x.ctypes.data for x in xs])
    pin, pout, pfl = arr(ds), arr(outs), arr(flags)
    lib.orc_fuse(V, _p(K), _p(R), _p(t), _p(W), _p(H), pin, float(tau), pout, pfl)
    return outs, flags


def rgb_to_lab(rgb) -> np.ndarray:
    rgb = np.ascontiguousarray(rgb, dtype=np.float64).reshape(3)
    out = np.zeros(3)
    _load().orc_rgb_to_lab(_p(rgb), _p(out))
    return out


def slic_seeds(rgb: np.ndarray, GW: int, GH: int) -> np.ndarray:
    """Initial SLIC centres {L, a, b, x, y} per grid cell (lfd_slic_oracle.c)."""
    rgb = np.ascontiguousarray(rgb, dtype=np.float64)
    H, W = rgb.shape[:2]
    c = np.zeros((GH * GW, 5))
    _load().orc_slic_seeds(W, H, _p(rgb), GW, GH, _p(c))
    return c


def slic_assign(rgb: np.ndarray, GW: int, GH: int, centres: np.ndarray, m: float):
    """One SLIC assignment: (labels (H, W) int32, near-tie flags (H, W))."""
    rgb = np.ascontiguousarray(rgb, dtype=np.float64)
    H, W = rgb.shape[:2]
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    lab = np.zeros((H, W), np.int32)
    fl = np.zeros((H, W), np.uint8)
    _load().orc_slic_assign(W, H, _p(rgb), GW, GH, _p(centres), float(m), _p(lab), _p(fl))
    return lab, fl


def slic_update(rgb: np.ndarray, GW: int, GH: int, labels: np.ndarray, centres: np.ndarray) -> np.ndarray:
    rgb = np.ascontiguousarray(rgb, dtype=np.float64)
    H, W = rgb.shape[:2]
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    out = np.zeros_like(centres)
    _load().orc_slic_update(W, H, _p(rgb), GW, GH, _p(labels), _p(centres), _p(out))
    return out


def slic(rgb: np.ndarray, GW: int, GH: int, m: float = 10.0, iterations: int = 10):
    """Full SLIC (seeds, iterations x (assign, update), final assign): (labels, centres)."""
    rgb = np.ascontiguousarray(rgb, dtype=np.float64)
    H, W = rgb.shape[:2]
    lab = np.zeros((H, W), np.int32)
    c = np.zeros((GH * GW, 5))
    _load().orc_slic(W, H, _p(rgb), GW, GH, float(m), int(iterations), _p(lab), _p(c))
    return lab, c


def terms_to_dict(t: Terms, n: int) -> dict:
    d = {k: getattr(t, k) for k in ("E", "Es", "Ec", "tssd", "E_lo", "E_hi", "Ec_lo", "Ec_hi",
                                      "tssd_lo", "tssd_hi", "flag_tssd", "flag_energy", "nviews")}
    for k in ("S", "Vt", "O", "S_lo", "S_hi", "V_lo", "V_hi", "O_lo", "O_hi", "nvalid", "nx", "ny", "nflag"):
        d[k] = np.array(list(getattr(t, k))[:n])
    return d


class Oracle:
    """FP64 reference of the method on one light field.

    K, R: (V,3,3); t: (V,3); rgb: (V,H,W,3) float in [0,1]; labels: (V,H,W) int32;
    GW, GH: superpixel grid size (ints or per-view sequences); params: dict with
    d_min, d_max, num_labels, T, sigma, alpha, eta, kernel_size_init,
    kernel_step_sp, max_neighbor_views, depth_domain, jitter, term_mask,
    sweep_frame, seed, lf_index, xy_eps, warm_iter_offset."""

    def __init__(self, K, R, t, rgb, labels, GW, GH, params: dict, threads: int | None = None,
                 margin_px: float = 1e-4, margin_rel: float = 1e-5):
        self.lib = _load()
        V = len(K)
        self.V = V
        rgb = [np.ascontiguousarray(np.asarray(r, dtype=np.float64)) for r in rgb]
        labels = [np.ascontiguousarray(np.asarray(l, dtype=np.int32)) for l in labels]
        self.H = np.array([r.shape[0] for r in rgb], dtype=np.int32)
        self.W = np.array([r.shape[1] for r in rgb], dtype=np.int32)
        gw = np.broadcast_to(np.asarray(GW, dtype=np.int32), (V,)).copy()
        gh = np.broadcast_to(np.asarray(GH, dtype=np.int32), (V,)).copy()
        for v in range(V):
            if labels[v].shape != rgb[v].shape[:2]:
                raise ValueError("label map and view size differ")
            if labels[v].size and (labels[v].min() < 0 or labels[v].max() >= gw[v] * gh[v]):
                raise ValueError("label outside the superpixel grid")
        self._keep = dict(
            W=self.W, H=self.H, GW=gw, GH=gh,
            K=np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(V, 9)),
            R=np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(V, 9)),
            t=np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(V, 3)),
            rgb=np.concatenate([r.reshape(-1) for r in rgb]),
            labels=np.concatenate([l.reshape(-1) for l in labels]),
        )
        self.GW, self.GH = gw, gh
        self.params = dict(params)
        inp = _Input()
        inp.V = V
        for k in ("W", "H", "GW", "GH", "K", "R", "t", "rgb", "labels"):
            setattr(inp, k, _p(self._keep[k]))
        inp.d_min = float(params["d_min"])
        inp.d_max = float(params["d_max"])
        inp.L = int(params["num_labels"])
        inp.T = float(params["T"])
        inp.sigma = float(params["sigma"])
        inp.alpha = float(params["alpha"])
        inp.eta = float(params["eta"])
        inp.kernel_size_init = int(params["kernel_size_init"])
        inp.kernel_step_sp = float(params["kernel_step_sp"])
        inp.max_neighbor_views = int(params["max_neighbor_views"])
        inp.depth_domain = int(params["depth_domain"])
        inp.jitter = int(params["jitter"])
        inp.term_mask = int(params["term_mask"])
        inp.sweep_frame = int(params["sweep_frame"])
        inp.seed = int(params["seed"]) & 0xFFFFFFFFFFFFFFFF
        inp.lf_index = int(params["lf_index"])
        inp.perturb_samples = int(params.get("perturb_samples", 0))
        inp.perturb_scale = float(params.get("perturb_scale", 0.05))
        inp.xy_eps = float(params["xy_eps"])
        inp.warm_iter_offset = int(params["warm_iter_offset"])
        inp.threads = int(threads or os.cpu_count() or 1)
        inp.margin_px = margin_px
        inp.margin_rel = margin_rel
        self._inp = inp
        self.h = self.lib.orc_create(C.byref(inp))
        if not self.h:
            raise ValueError("oracle rejected the input")
        self.S = np.array([self.lib.orc_num_sp(self.h, v) for v in range(V)], dtype=np.int64)
        self.sp_base = np.array([self.lib.orc_sp_base(self.h, v) for v in range(V)], dtype=np.int64)
        self.S_total = int(self.S.sum())
        self.sigma = float(self.lib.orc_sigma(self.h))
        self.delta = float(self.lib.orc_delta(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    # ---- superpixels / host logic ----
    def sp_stats(self, v: int) -> dict:
        S = int(self.S[v])
        n = int(self.W[v]) * int(self.H[v])
        cnt = np.zeros(S, np.int64)
        cen = np.zeros((S, 2))
        col = np.zeros((S, 3))
        minw = np.zeros(S)
        off = np.zeros(S + 1, np.int32)
        pix = np.zeros(n, np.int32)
        self.lib.orc_sp_stats(self.h, v, _p(cnt), _p(cen), _p(col), _p(minw), _p(off), _p(pix))
        return dict(cnt=cnt, cen=cen, col=col, minw=minw, off=off, pix=pix)

    def neighbor_views(self, v: int) -> np.ndarray:
        out = np.zeros(MAXN, np.int32)
        n = self.lib.orc_neighbor_views(self.h, v, _p(out))
        return out[:n].copy()

    def kernel_params(self, v: int):
        a = np.zeros(1, np.int32)
        b = np.zeros(1, np.int32)
        self.lib.orc_kernel_params(self.h, v, _p(a), _p(b))
        return int(a[0]), int(b[0])

    def plane_depth(self, v, plane, centroid, u, vv) -> float:
        return float(self.lib.orc_plane_depth(self.h, v, *map(float, plane), float(centroid[0]), float(centroid[1]),
                                              float(u), float(vv)))

    def project_pixel(self, v, k, plane, centroid, u, vv):
        out = np.zeros(3)
        ok = self.lib.orc_project_pixel(self.h, v, k, *map(float, plane), float(centroid[0]), float(centroid[1]),
                                        float(u), float(vv), _p(out))
        return bool(ok), out

    # ---- method steps ----
    def _items(self, items):
        if items is None:
            return None, self.S_total
        it = np.ascontiguousarray(np.asarray(items, dtype=np.int32))
        return it, len(it)

    def sweep(self, items=None, want_costs: bool = False):
        it, n = self._items(items)
        planes = np.zeros((self.S_total, 4))
        lab = np.zeros(n, np.int32)
        L = int(self.params["num_labels"])
        cost = lo = hi = None
        if want_costs:
            cost, lo, hi = (np.zeros((n, L)) for _ in range(3))
        self.lib.orc_sweep(self.h, None if it is None else _p(it), n, _p(planes), _p(lab),
                           None if cost is None else _p(cost), None if lo is None else _p(lo),
                           None if hi is None else _p(hi))
        return dict(planes=planes, label=lab, cost=cost, cost_lo=lo, cost_hi=hi)

    def rasterize(self, planes: np.ndarray):
        planes = np.ascontiguousarray(planes, dtype=np.float64).reshape(-1)
        tot = int(np.sum(self.W.astype(np.int64) * self.H))
        maps = np.zeros(tot)
        depth = np.zeros(tot)
        self.lib.orc_rasterize(self.h, _p(planes), _p(maps), _p(depth))
        out_m, out_d, o = [], [], 0
        for v in range(self.V):
            n = int(self.W[v]) * int(self.H[v])
            out_m.append(maps[o:o + n].reshape(self.H[v], self.W[v]))
            out_d.append(depth[o:o + n].reshape(self.H[v], self.W[v]))
            o += n
        return out_m, out_d

    def iterate(self, it_index: int, planes_in: np.ndarray, items=None, cand_cap: int = 0):
        planes_in = np.ascontiguousarray(planes_in, dtype=np.float64).reshape(self.S_total, 4)
        it, n = self._items(items)
        out = np.zeros_like(planes_in)
        choice = np.zeros((n, 2), np.int32)
        energy = np.zeros((n, 2))
        flag = np.zeros(n, np.int32)
        cand = np.zeros((n, max(cand_cap, 1), 3)) if cand_cap > 0 else None
        ref = np.zeros((n, REF_MAX, 3))
        self.lib.orc_iterate(self.h, it_index, _p(planes_in), None if it is None else _p(it), n, _p(out),
                             _p(choice), _p(energy), _p(flag), None if cand is None else _p(cand), cand_cap, _p(ref))
        return dict(planes=out, choice=choice, energy=energy, flag=flag, cand=cand, ref=ref)

    def refine_candidates(self, planes_state: np.ndarray, gsp: int, dnew: float, normal=None,
                          it_index: int = 1) -> np.ndarray:
        """Energies (E, lo, hi) of the refinement candidates of superpixel gsp at
        depth dnew: the 8 ring triangles, then the perturbation samples of the
        plane (dnew, normal) when the variant is on.  Shape (REF_MAX, 3)."""
        planes_state = np.ascontiguousarray(planes_state, dtype=np.float64).reshape(-1)
        out = np.zeros((REF_MAX, 3))
        n = np.zeros(3) if normal is None else np.asarray(normal, dtype=np.float64)
        self.lib.orc_refine_candidates(self.h, _p(planes_state), int(gsp), float(dnew), float(n[0]), float(n[1]),
                                       float(n[2]), int(it_index), _p(out))
        return out

    def score(self, planes_state: np.ndarray, queries) -> list:
        """queries: iterable of (view, sp, d, nx, ny, nz).  Returns a list of dicts."""
        planes_state = np.ascontiguousarray(planes_state, dtype=np.float64).reshape(-1)
        qs = list(queries)
        arr = (Query * max(len(qs), 1))()
        for i, q in enumerate(qs):
            arr[i] = Query(int(q[0]), int(q[1]), *map(float, q[2:6]))
        out = (Terms * max(len(qs), 1))()
        self.lib.orc_score(self.h, _p(planes_state), C.cast(arr, C.c_void_p), len(qs), C.cast(out, C.c_void_p))
        res = []
        for i, q in enumerate(qs):
            res.append(terms_to_dict(out[i], out[i].nviews))
        return res

    def run(self, iterations: int | None = None, planes0=None):
        """Full frame: sweep (unless planes0 given) then `iterations` Jacobi iterations."""
        its = int(self.params.get("iterations", 4) if iterations is None else iterations)
        planes = self.sweep()["planes"] if planes0 is None else np.array(planes0, dtype=np.float64)
        hist = [planes]
        for i in range(1, its + 1):
            planes = self.iterate(i, planes)["planes"]
            hist.append(planes)
        return planes, hist
