"""Python binding of liblfdepth (include/lfdepth.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts torch
tensors (device memory, streams) and numpy camera arrays into the C ABI's
plain pointers and sizes.  Importing it loads the library and fails loudly if
it is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

_lib = None

MAX_NEIGHBOR_VIEWS = 8
TERMS_HEAD = 4
TERMS_PER_VIEW = 6
TERMS_STRIDE = TERMS_HEAD + MAX_NEIGHBOR_VIEWS * TERMS_PER_VIEW

LFD_ERR_BUDGET = 4
LFD_ERR_TIMEOUT = 5
LFD_ERR_BUSY = 7

FMT = {"rgba8": 0, "rgba_f16": 1, "rgba_bf16": 2, "rgba_f32": 3}
_DTYPE_FMT = {torch.uint8: 0, torch.float16: 1, torch.bfloat16: 2, torch.float32: 3}
_TEXEL = {0: 4, 1: 8, 2: 8, 3: 16}


class Camera(C.Structure):
    _fields_ = [("K", C.c_double * 9), ("R", C.c_double * 9), ("t", C.c_double * 3),
                ("width", C.c_int32), ("height", C.c_int32)]


class LightFieldC(C.Structure):
    _fields_ = [("num_views", C.c_int32), ("fmt", C.c_int32), ("cams", C.POINTER(Camera)),
                ("views", C.POINTER(C.c_void_p)), ("view_pitch_bytes", C.POINTER(C.c_int64)),
                ("labels", C.POINTER(C.c_void_p)), ("grid_w", C.POINTER(C.c_int32)),
                ("grid_h", C.POINTER(C.c_int32))]


class Params(C.Structure):
    _fields_ = [("d_min", C.c_double), ("d_max", C.c_double), ("num_labels", C.c_int32),
                ("iterations", C.c_int32), ("T", C.c_double), ("sigma", C.c_double), ("alpha", C.c_double),
                ("eta", C.c_double), ("kernel_size_init", C.c_int32), ("kernel_step_sp", C.c_double),
                ("max_neighbor_views", C.c_int32), ("depth_domain", C.c_int32), ("jitter", C.c_int32),
                ("term_mask", C.c_uint32), ("sweep_frame", C.c_int32), ("seed", C.c_uint64),
                ("lf_index", C.c_int32), ("xy_eps", C.c_double), ("warm_iter_offset", C.c_int32),
                ("perturb_samples", C.c_int32), ("perturb_scale", C.c_double)]


class Query(C.Structure):
    _fields_ = [("view", C.c_int32), ("sp", C.c_int32), ("d", C.c_float), ("nx", C.c_float),
                ("ny", C.c_float), ("nz", C.c_float)]


class BatchOptions(C.Structure):
    _fields_ = [("autotune", C.c_int32), ("graph", C.c_int32), ("sweep_threads", C.c_int32),
                ("sweep_persistent", C.c_int32), ("prop_blocks", C.c_int32), ("prop_persistent", C.c_int32),
                ("prop_batch", C.c_int32), ("order_bands", C.c_int32), ("prop_coop", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("req_id", C.c_uint64), ("rig_id", C.c_int32), ("warm", C.c_int32), ("frame", C.c_int64),
                ("submit_ns", C.c_int64), ("done_ns", C.c_int64), ("status", C.c_int32), ("slot", C.c_int32),
                ("start_ns", C.c_int64), ("batch", C.c_int32), ("reserved", C.c_int32)]


class LfdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lfdepth status {status}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblfdepth.so (building it first when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"liblfdepth.so not built at {path}")
        _build.build()
    lib = C.CDLL(path)
    vp, i32 = C.c_void_p, C.c_int32
    P = C.POINTER
    lib.lfd_version.restype = i32
    lib.lfd_struct_sizes.argtypes = [P(i32)]
    lib.lfd_status_string.restype = C.c_char_p
    lib.lfd_status_string.argtypes = [i32]
    lib.lfd_last_error.restype = C.c_char_p
    lib.lfd_last_error.argtypes = [vp]
    lib.lfd_params_default.argtypes = [P(Params)]
    lib.lfd_create.argtypes = [P(vp), i32, C.c_uint64]
    lib.lfd_destroy.argtypes = [vp]
    lib.lfd_set_input.argtypes = [vp, P(LightFieldC), P(Params), vp]
    lib.lfd_num_superpixels.argtypes = [vp, i32, P(i32)]
    lib.lfd_plane_sweep.argtypes = [vp, P(vp), P(vp), P(vp), vp]
    lib.lfd_rasterize.argtypes = [vp, P(vp), P(vp), vp]
    lib.lfd_iterate.argtypes = [vp, i32, P(vp), P(vp), P(vp), P(vp), vp]
    lib.lfd_estimate.argtypes = [vp, P(LightFieldC), P(Params), P(vp), P(vp), P(vp), vp]
    lib.lfd_estimate_host.argtypes = [vp, P(LightFieldC), P(Params), P(vp), P(vp), vp]
    lib.lfd_synchronize.argtypes = [vp, vp]
    lib.lfd_counters.argtypes = [vp, P(C.c_uint64), P(C.c_uint64), vp]
    lib.lfd_score.argtypes = [vp, P(vp), i32, P(Query), P(C.c_float), vp]
    lib.lfd_get_superpixels.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    lib.lfd_neighbor_views.argtypes = [P(Camera), i32, i32, P(i32), P(i32)]
    lib.lfd_profile_enable.argtypes = [vp, i32]
    lib.lfd_profile_read.argtypes = [vp, P(C.c_double), P(C.c_int64)]
    lib.lfd_superpixel_stats_noalloc.argtypes = [vp, vp, i32, i32, C.c_int64, i32, i32, i32, C.c_double, vp, vp]
    lib.lfd_superpixel_stats_noalloc.restype = i32
    lib.lfd_kernel_offsets.restype = i32
    lib.lfd_kernel_offsets.argtypes = [i32, i32, i32, P(i32), i32]
    lib.lfd_batch_options_default.argtypes = [P(BatchOptions)]
    lib.lfd_batch_options_default.restype = None
    lib.lfd_estimate_batch.argtypes = [vp, i32, P(LightFieldC), P(Params), P(vp), P(vp), P(BatchOptions), vp]
    lib.lfd_estimate_batch_warm.argtypes = [vp, i32, P(LightFieldC), P(Params), P(vp), P(vp), P(vp),
                                            P(BatchOptions), vp]
    lib.lfd_launch_config.argtypes = [vp, P(i32)]
    lib.lfd_set_pair_forms.argtypes = [vp, i32]
    lib.lfd_pair_form.argtypes = [vp, P(i32)]
    lib.lfd_workspace_required.argtypes = [i32, P(LightFieldC), P(C.c_uint64)]
    lib.lfd_fuse.argtypes = [vp, P(vp), P(vp), C.c_double, vp]
    lib.lfd_slic.argtypes = [vp, i32, P(vp), vp, i32, vp, vp, vp, vp, C.c_double, i32, P(vp), P(vp), P(vp), vp]
    lib.lfd_server_create.argtypes = [P(vp), i32, C.c_uint64, i32]
    lib.lfd_server_destroy.argtypes = [vp]
    lib.lfd_server_last_error.argtypes = [vp]
    lib.lfd_server_last_error.restype = C.c_char_p
    lib.lfd_server_configure.argtypes = [vp, i32, i32, i32]
    lib.lfd_server_now_ns.argtypes = []
    lib.lfd_server_now_ns.restype = C.c_int64
    lib.lfd_server_submit.argtypes = [vp, i32, P(LightFieldC), P(Params), P(vp), P(vp), P(C.c_uint64)]
    lib.lfd_server_poll.argtypes = [vp, C.c_uint64, i32, P(Result)]
    lib.lfd_server_set_max_batch.argtypes = [vp, i32]
    lib.lfd_server_stats.argtypes = [vp, P(C.c_int64), P(C.c_int64)]
    lib.lfd_server_export_state.argtypes = [vp, i32, vp, C.c_int64, P(C.c_int64)]
    lib.lfd_server_import_state.argtypes = [vp, i32, vp, C.c_int64]
    for name in ("lfd_create", "lfd_destroy", "lfd_set_input", "lfd_num_superpixels", "lfd_plane_sweep",
                 "lfd_rasterize", "lfd_iterate", "lfd_estimate", "lfd_estimate_host", "lfd_synchronize",
                 "lfd_counters", "lfd_score", "lfd_get_superpixels", "lfd_neighbor_views", "lfd_profile_enable",
                 "lfd_profile_read", "lfd_estimate_batch", "lfd_estimate_batch_warm", "lfd_launch_config", "lfd_set_pair_forms", "lfd_pair_form", "lfd_workspace_required", "lfd_fuse", "lfd_slic",
                 "lfd_server_create", "lfd_server_destroy", "lfd_server_configure", "lfd_server_submit",
                 "lfd_server_poll", "lfd_server_export_state", "lfd_server_import_state", "lfd_server_set_max_batch",
                 "lfd_server_stats"):
        getattr(lib, name).restype = i32
    sizes = (i32 * 8)()
    lib.lfd_struct_sizes(sizes)
    want = [C.sizeof(Camera), C.sizeof(LightFieldC), C.sizeof(Params), C.sizeof(Query), C.sizeof(BatchOptions),
            C.sizeof(Result)]
    if list(sizes)[:6] != want:
        raise RuntimeError(f"lfdepth ABI mismatch: library struct sizes {list(sizes)} != binding {want}")
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# host-logic entry points (no GPU needed)
# ---------------------------------------------------------------------------

def make_cameras(K, R, t, W, H):
    V = len(K)
    cams = (Camera * V)()
    for v in range(V):
        cams[v].K[:] = [float(x) for x in np.asarray(K[v], dtype=np.float64).reshape(9)]
        cams[v].R[:] = [float(x) for x in np.asarray(R[v], dtype=np.float64).reshape(9)]
        cams[v].t[:] = [float(x) for x in np.asarray(t[v], dtype=np.float64).reshape(3)]
        cams[v].width = int(W if np.isscalar(W) else W[v])
        cams[v].height = int(H if np.isscalar(H) else H[v])
    return cams


def neighbor_views(K, R, t, W, H, max_k: int = 0) -> np.ndarray:
    lib = load()
    cams = make_cameras(K, R, t, W, H)
    V = len(K)
    out = (C.c_int32 * (V * MAX_NEIGHBOR_VIEWS))()
    k = C.c_int32()
    st = lib.lfd_neighbor_views(cams, V, max_k, out, C.byref(k))
    if st != 0:
        raise LfdError(st, lib.lfd_status_string(st).decode())
    return np.array(out, dtype=np.int32).reshape(V, MAX_NEIGHBOR_VIEWS)[:, :k.value]


def kernel_offsets(size_init: int, steps_init: int, it: int) -> np.ndarray:
    lib = load()
    n = lib.lfd_kernel_offsets(size_init, steps_init, it, None, 0)
    buf = (C.c_int32 * (2 * n))()
    lib.lfd_kernel_offsets(size_init, steps_init, it, buf, n)
    return np.array(buf, dtype=np.int32).reshape(n, 2)


def superpixel_stats_noalloc(labels: torch.Tensor, image: torch.Tensor, grid_w: int, grid_h: int, alpha: float,
                             stats_out: torch.Tensor, stream=None) -> None:
    """lfd_superpixel_stats_noalloc on one view: labels (H,W) int32 and image
    (H,W,4) texels on the device, stats_out (grid_w*grid_h, 8) float32 on the
    device.  The image may have padded rows (row stride >= W texels); its
    texels must be packed within a row.  Raises ValueError for arguments the
    call cannot take safely, LfdError for a status other than LFD_OK."""
    lib = load()
    if not (isinstance(labels, torch.Tensor) and isinstance(image, torch.Tensor) and isinstance(stats_out, torch.Tensor)):
        raise ValueError("labels, image and stats_out must be torch tensors")
    if not (labels.is_cuda and image.is_cuda and stats_out.is_cuda):
        raise ValueError("labels, image and stats_out must be CUDA tensors")
    if not (labels.device == image.device == stats_out.device):
        raise ValueError("labels, image and stats_out must be on one device")
    if labels.dtype != torch.int32 or labels.dim() != 2 or not labels.is_contiguous():
        raise ValueError("labels must be a contiguous (H, W) int32 tensor")
    H, W = int(labels.shape[0]), int(labels.shape[1])
    if image.dtype not in _DTYPE_FMT or image.dim() != 3 or tuple(image.shape) != (H, W, 4):
        raise ValueError(f"image must be (H, W, 4) = ({H}, {W}, 4) of uint8/float16/bfloat16/float32")
    if image.stride(2) != 1 or image.stride(1) != 4 or image.stride(0) < 4 * W:
        raise ValueError("image texels must be packed within each row (strides (>= 4W, 4, 1))")
    if stats_out.dtype != torch.float32 or not stats_out.is_contiguous() or \
            stats_out.numel() < int(grid_w) * int(grid_h) * 8:
        raise ValueError("stats_out must be a contiguous float32 tensor of at least grid_w * grid_h * 8 elements")
    fmt = _DTYPE_FMT[image.dtype]
    pitch = image.stride(0) * image.element_size()
    st = lib.lfd_superpixel_stats_noalloc(labels.data_ptr(), image.data_ptr(), W, H, pitch, fmt,
                                          int(grid_w), int(grid_h), float(alpha), stats_out.data_ptr(),
                                          _stream(stream))
    if st != 0:
        raise LfdError(st, f"lfd_superpixel_stats_noalloc: {lib.lfd_status_string(st).decode()}")


def params_struct(params: dict) -> Params:
    p = Params()
    load().lfd_params_default(C.byref(p))
    for k, v in params.items():
        if k in dict(Params._fields_):
            setattr(p, k, v if not isinstance(v, (np.integer, np.floating)) else v.item())
    return p


def _ptr_array(ptrs):
    arr = (C.c_void_p * len(ptrs))()
    for i, q in enumerate(ptrs):
        arr[i] = q
    return arr


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def marshal_lightfield(views, labels, K, R, t, GW, GH):
    """lfd_lightfield of device tensors views (V,H,W,4) and labels (V,H,W) int32;
    returns it with the ctypes arrays and tensors it points into (keep alive)."""
    V = len(K)
    assert views.dim() == 4 and views.shape[0] == V and views.shape[-1] == 4
    fmt = _DTYPE_FMT[views.dtype]
    H, W = int(views.shape[1]), int(views.shape[2])
    cams = make_cameras(K, R, t, W, H)
    vptr = _ptr_array([views[v].data_ptr() for v in range(V)])
    lptr = _ptr_array([labels[v].data_ptr() for v in range(V)])
    pitch = (C.c_int64 * V)(*([W * _TEXEL[fmt]] * V))
    gw = (C.c_int32 * V)(*([int(GW)] * V if np.isscalar(GW) else [int(x) for x in GW]))
    gh = (C.c_int32 * V)(*([int(GH)] * V if np.isscalar(GH) else [int(x) for x in GH]))
    lf = LightFieldC(V, fmt, cams, vptr, pitch, lptr, gw, gh)
    keep = (cams, vptr, lptr, pitch, gw, gh, views, labels)
    return lf, keep


class Context:
    """One light-field workspace on one GPU (lfd_ctx)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.lib = load()
        self.h = C.c_void_p()
        self._check(self.lib.lfd_create(C.byref(self.h), device, hbm_budget), "lfd_create")
        self.device = device
        self._keep = []
        self.V = 0
        self.S = np.zeros(0, np.int64)
        self.sp_base = np.zeros(0, np.int64)
        self.S_total = 0

    def close(self):
        if self.h:
            self.lib.lfd_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != 0:
            msg = self.lib.lfd_last_error(self.h).decode() if self.h else ""
            raise LfdError(st, f"{what}: {self.lib.lfd_status_string(st).decode()}: {msg}")

    # -- marshalling ---------------------------------------------------------
    def _lightfield(self, views, labels, K, R, t, GW, GH):
        return marshal_lightfield(views, labels, K, R, t, GW, GH)

    def _layout(self, V, GW, GH):
        gw = [int(GW)] * V if np.isscalar(GW) else [int(x) for x in GW]
        gh = [int(GH)] * V if np.isscalar(GH) else [int(x) for x in GH]
        self.S = np.array([a * b for a, b in zip(gw, gh)], dtype=np.int64)
        self.sp_base = np.concatenate([[0], np.cumsum(self.S)[:-1]]).astype(np.int64)
        self.S_total = int(self.S.sum())
        self.V = V
        self.view_hw = None

    def _view_ptrs(self, flat: torch.Tensor, per_sp: int):
        assert flat.is_cuda and flat.is_contiguous()
        if self.V == 0:                      # nothing bound: the library reports the call order
            return _ptr_array([flat.data_ptr()])
        es = flat.element_size()
        base = flat.data_ptr()
        return _ptr_array([base + int(self.sp_base[v]) * per_sp * es for v in range(self.V)])

    # -- staged hot path -----------------------------------------------------
    def set_input(self, views, labels, K, R, t, GW, GH, params: dict, stream=None):
        """views: (V,H,W,4) cuda tensor (uint8 / float16 / bfloat16 / float32);
        labels: (V,H,W) int32 cuda tensor."""
        lf, keep = self._lightfield(views, labels, K, R, t, GW, GH)
        self._layout(len(K), GW, GH)
        self.H, self.W = int(views.shape[1]), int(views.shape[2])
        p = params_struct(params)
        self._keep = [keep, p]
        self._check(self.lib.lfd_set_input(self.h, C.byref(lf), C.byref(p), _stream(stream)), "lfd_set_input")
        self.params = dict(params)

    def plane_sweep(self, want_labels: bool = False, want_costs: bool = False, stream=None):
        dev = torch.device("cuda", self.device)
        planes = torch.zeros((self.S_total, 4), dtype=torch.float32, device=dev)
        labels = torch.zeros(self.S_total, dtype=torch.int32, device=dev) if want_labels else None
        L = int(self.params["num_labels"])
        costs = torch.zeros((self.S_total, L), dtype=torch.float32, device=dev) if want_costs else None
        self._check(self.lib.lfd_plane_sweep(
            self.h, self._view_ptrs(planes, 4),
            self._view_ptrs(labels, 1) if labels is not None else None,
            self._view_ptrs(costs, L) if costs is not None else None, _stream(stream)), "lfd_plane_sweep")
        return planes, labels, costs

    def rasterize(self, planes: torch.Tensor, want_depth: bool = True, stream=None):
        dev = planes.device
        depth = torch.zeros((self.V, self.H, self.W), dtype=torch.float32, device=dev) if want_depth else None
        dptr = _ptr_array([depth[v].data_ptr() for v in range(self.V)]) if want_depth else None
        self._check(self.lib.lfd_rasterize(self.h, self._view_ptrs(planes.contiguous(), 4), dptr, _stream(stream)),
                    "lfd_rasterize")
        return depth

    def iterate(self, it: int, planes_in: torch.Tensor, want_choice: bool = False, stream=None):
        planes_in = planes_in.contiguous()
        out = torch.empty_like(planes_in)
        choice = torch.zeros((self.S_total, 2), dtype=torch.int32, device=planes_in.device) if want_choice else None
        energy = torch.zeros((self.S_total, 2), dtype=torch.float32, device=planes_in.device) if want_choice else None
        self._check(self.lib.lfd_iterate(
            self.h, it, self._view_ptrs(planes_in, 4), self._view_ptrs(out, 4),
            self._view_ptrs(choice, 2) if choice is not None else None,
            self._view_ptrs(energy, 2) if energy is not None else None, _stream(stream)), "lfd_iterate")
        return out, choice, energy

    def estimate(self, views, labels, K, R, t, GW, GH, params: dict, warm=None, want_depth: bool = True,
                 out_planes=None, out_depth=None, stream=None):
        lf, keep = self._lightfield(views, labels, K, R, t, GW, GH)
        self._layout(len(K), GW, GH)
        self.H, self.W = int(views.shape[1]), int(views.shape[2])
        p = params_struct(params)
        self.params = dict(params)
        dev = views.device
        planes = out_planes if out_planes is not None else torch.zeros((self.S_total, 4), dtype=torch.float32, device=dev)
        depth = None
        dptr = None
        if want_depth:
            depth = out_depth if out_depth is not None else torch.zeros((self.V, self.H, self.W), dtype=torch.float32, device=dev)
            dptr = _ptr_array([depth[v].data_ptr() for v in range(self.V)])
        wptr = self._view_ptrs(warm.contiguous(), 4) if warm is not None else None
        pp = self._view_ptrs(planes, 4)
        self._keep = [keep, p, wptr, pp, dptr, warm]
        self._check(self.lib.lfd_estimate(self.h, C.byref(lf), C.byref(p), wptr, pp, dptr, _stream(stream)),
                    "lfd_estimate")
        return planes, depth

    def estimate_host(self, views_host: torch.Tensor, labels_host: torch.Tensor, K, R, t, GW, GH, params: dict,
                      planes_host: torch.Tensor, depth_host: torch.Tensor | None, stream=None):
        """Whole frame through lfd_estimate_host: inputs and outputs in (pinned) host memory."""
        V = len(K)
        self._layout(V, GW, GH)
        self.H, self.W = int(views_host.shape[1]), int(views_host.shape[2])
        fmt = _DTYPE_FMT[views_host.dtype]
        cams = make_cameras(K, R, t, self.W, self.H)
        vptr = _ptr_array([views_host[v].data_ptr() for v in range(V)])
        lptr = _ptr_array([labels_host[v].data_ptr() for v in range(V)])
        pitch = (C.c_int64 * V)(*([self.W * _TEXEL[fmt]] * V))
        gw = (C.c_int32 * V)(*([int(GW)] * V))
        gh = (C.c_int32 * V)(*([int(GH)] * V))
        lf = LightFieldC(V, fmt, cams, vptr, pitch, lptr, gw, gh)
        p = params_struct(params)
        self.params = dict(params)
        base = planes_host.data_ptr()
        pp = _ptr_array([base + int(self.sp_base[v]) * 16 for v in range(V)])
        dptr = _ptr_array([depth_host[v].data_ptr() for v in range(V)]) if depth_host is not None else None
        self._keep = [cams, vptr, lptr, pitch, gw, gh, p, pp, dptr]
        self._check(self.lib.lfd_estimate_host(self.h, C.byref(lf), C.byref(p), pp, dptr, _stream(stream)),
                    "lfd_estimate_host")

    def estimate_batch(self, items, options: dict | None = None, want_depth: bool = True, out=None,
                       stream=None, warm=None):
        """Several light fields in one pass (lfd_estimate_batch, or
        lfd_estimate_batch_warm when `warm` is given).

        items: list of dicts with keys views, labels, K, R, t, GW, GH, params
        (as for `estimate`).  options: lfd_batch_options fields.  out: the
        (planes, depths) returned by an earlier call with the same items, to
        write into the same buffers (a graph replay needs identical pointers).
        warm: None, or a list with one entry per item: None (cold) or a
        (S_l, 4) float32 cuda tensor of that light field's warm planes.
        Returns (planes, depths): planes (S_total, 4) over all light fields'
        superpixels in order; depths a list of (V_l, H_l, W_l) tensors or None."""
        n = len(items)
        lfs = (LightFieldC * n)()
        ps = (Params * n)()
        keep = []
        S_all, V_all = [], 0
        for l, it in enumerate(items):
            lf, k = self._lightfield(it["views"], it["labels"], it["K"], it["R"], it["t"], it["GW"], it["GH"])
            lfs[l] = lf
            ps[l] = params_struct(it["params"])
            keep.append(k)
            V = len(it["K"])
            gw = [int(it["GW"])] * V if np.isscalar(it["GW"]) else [int(x) for x in it["GW"]]
            gh = [int(it["GH"])] * V if np.isscalar(it["GH"]) else [int(x) for x in it["GH"]]
            S_all += [a * b for a, b in zip(gw, gh)]
            V_all += V
        self.S = np.array(S_all, dtype=np.int64)
        self.sp_base = np.concatenate([[0], np.cumsum(self.S)[:-1]]).astype(np.int64)
        self.S_total = int(self.S.sum())
        self.V = V_all
        self.H, self.W = int(items[0]["views"].shape[1]), int(items[0]["views"].shape[2])
        self.view_hw = [(int(it["views"].shape[1]), int(it["views"].shape[2])) for it in items
                        for _ in range(len(it["K"]))]
        self.params = dict(items[0]["params"])
        dev = items[0]["views"].device
        if out is not None:
            planes, depths = out
        else:
            planes = torch.zeros((self.S_total, 4), dtype=torch.float32, device=dev)
            depths = [torch.zeros((len(it["K"]), int(it["views"].shape[1]), int(it["views"].shape[2])),
                                  dtype=torch.float32, device=dev) for it in items] if want_depth else None
        pp_all = self._view_ptrs(planes, 4)
        pp = (C.c_void_p * n)()
        dd = (C.c_void_p * n)()
        g = 0
        for l, it in enumerate(items):
            V = len(it["K"])
            arr = _ptr_array([pp_all[g + v] for v in range(V)])
            pp[l] = C.cast(arr, C.c_void_p)
            keep.append(arr)
            if depths is not None:
                darr = _ptr_array([depths[l][v].data_ptr() for v in range(V)])
                dd[l] = C.cast(darr, C.c_void_p)
                keep.append(darr)
            g += V
        o = BatchOptions()
        self.lib.lfd_batch_options_default(C.byref(o))
        for key, val in (options or {}).items():
            setattr(o, key, int(val))
        self._keep = [keep, lfs, ps, pp_all, pp, dd, o, planes, depths]
        if warm is None:
            self._check(self.lib.lfd_estimate_batch(self.h, n, lfs, ps, pp, dd if depths is not None else None,
                                                    C.byref(o), _stream(stream)), "lfd_estimate_batch")
            return planes, depths
        assert len(warm) == n, "one warm entry per light field"
        ww = (C.c_void_p * n)()
        for l, (it, wp) in enumerate(zip(items, warm)):
            if wp is None:
                continue
            wp = wp.contiguous()
            V = len(it["K"])
            S_l = [a * b for a, b in zip(*(([int(it[k])] * V if np.isscalar(it[k]) else [int(x) for x in it[k]])
                                             for k in ("GW", "GH")))]
            assert wp.is_cuda and wp.dtype == torch.float32 and wp.shape == (sum(S_l), 4)
            offs = np.concatenate([[0], np.cumsum(S_l)[:-1]])
            arr = _ptr_array([wp.data_ptr() + 16 * int(o_) for o_ in offs])
            ww[l] = C.cast(arr, C.c_void_p)
            keep += [arr, wp]
        self._keep.append(ww)
        self._check(self.lib.lfd_estimate_batch_warm(self.h, n, lfs, ps, ww, pp, dd if depths is not None else None,
                                                     C.byref(o), _stream(stream)), "lfd_estimate_batch_warm")
        return planes, depths

    def fuse(self, depth_in, tau: float = 0.01, stream=None):
        """Stability-based fusion (lfd_fuse) of one depth map per bound view:
        depth_in is a (V, H, W) float32 cuda tensor or a list of (H_v, W_v)
        tensors; returns the fused maps in the same form."""
        maps = [depth_in[v] for v in range(depth_in.shape[0])] if torch.is_tensor(depth_in) else list(depth_in)
        assert len(maps) == self.V, "one depth map per bound view"
        maps = [m.contiguous() for m in maps]
        if torch.is_tensor(depth_in):
            out = torch.zeros_like(depth_in)
            outs = [out[v] for v in range(self.V)]
        else:
            outs = [torch.zeros_like(m) for m in maps]
            out = outs
        pin = _ptr_array([m.data_ptr() for m in maps])
        pout = _ptr_array([o.data_ptr() for o in outs])
        self._keep = [self._keep, pin, pout, maps, outs]
        self._check(self.lib.lfd_fuse(self.h, pin, pout, float(tau), _stream(stream)), "lfd_fuse")
        return out

    def slic(self, views: torch.Tensor, GW: int, GH: int, compactness: float = 10.0, iterations: int = 10,
             centres_in: torch.Tensor | None = None, want_centres: bool = False, stream=None):
        """SLIC label maps (lfd_slic) of views (V, H, W, 4) on the device: returns
        labels (V, H, W) int32 and, with want_centres, centres (V, GW*GH, 5)."""
        V, H, W = int(views.shape[0]), int(views.shape[1]), int(views.shape[2])
        fmt = _DTYPE_FMT[views.dtype]
        labels = torch.zeros((V, H, W), dtype=torch.int32, device=views.device)
        cout = torch.zeros((V, GW * GH, 5), dtype=torch.float32, device=views.device) if want_centres else None
        vptr = _ptr_array([views[v].data_ptr() for v in range(V)])
        lptr = _ptr_array([labels[v].data_ptr() for v in range(V)])
        ci = _ptr_array([centres_in[v].data_ptr() for v in range(V)]) if centres_in is not None else None
        co = _ptr_array([cout[v].data_ptr() for v in range(V)]) if cout is not None else None
        ints = lambda x: (C.c_int32 * V)(*([int(x)] * V))
        w, h, gw, gh = ints(W), ints(H), ints(GW), ints(GH)
        self._keep = [self._keep, vptr, lptr, ci, co, w, h, gw, gh, views, centres_in]
        self._check(self.lib.lfd_slic(self.h, V, vptr, None, fmt, w, h, gw, gh, float(compactness), int(iterations),
                                      lptr, ci, co, _stream(stream)), "lfd_slic")
        return (labels, cout) if want_centres else labels

    def launch_config(self) -> dict:
        out = (C.c_int32 * 7)()
        self._check(self.lib.lfd_launch_config(self.h, out), "lfd_launch_config")
        return dict(sweep_threads=out[0], sweep_persistent=out[1], prop_blocks=out[2], prop_persistent=out[3],
                    prop_batch=out[4], order_bands=out[5], prop_coop=out[6])

    def set_pair_forms(self, max_form: int):
        """Largest homography specialisation (0 general, 1 affine, 2 translation)
        used for inputs bound after the call."""
        self._check(self.lib.lfd_set_pair_forms(self.h, int(max_form)), "lfd_set_pair_forms")

    def pair_form(self) -> int:
        """Specialisation of the bound input: 0 general, 1 affine, 2 translation."""
        out = C.c_int32()
        self._check(self.lib.lfd_pair_form(self.h, C.byref(out)), "lfd_pair_form")
        return int(out.value)

    def synchronize(self, stream=None):
        self._check(self.lib.lfd_synchronize(self.h, _stream(stream)), "lfd_synchronize")

    def counters(self, stream=None):
        a, b = C.c_uint64(), C.c_uint64()
        self._check(self.lib.lfd_counters(self.h, C.byref(a), C.byref(b), _stream(stream)), "lfd_counters")
        return int(a.value), int(b.value)

    STAGES = ("superpixels", "sweep", "raster", "propagate", "fusion")

    def profile_enable(self, on: bool = True):
        self._check(self.lib.lfd_profile_enable(self.h, 1 if on else 0), "lfd_profile_enable")

    def profile_read(self) -> dict:
        ms = (C.c_double * len(self.STAGES))()
        n = (C.c_int64 * len(self.STAGES))()
        self._check(self.lib.lfd_profile_read(self.h, ms, n), "lfd_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.STAGES)}

    def score(self, state_planes: torch.Tensor, queries) -> np.ndarray:
        qs = list(queries)
        arr = (Query * max(len(qs), 1))()
        for i, q in enumerate(qs):
            arr[i] = Query(int(q[0]), int(q[1]), *map(float, q[2:6]))
        out = np.zeros((max(len(qs), 1), TERMS_STRIDE), dtype=np.float32)
        self._check(self.lib.lfd_score(self.h, self._view_ptrs(state_planes.contiguous(), 4), len(qs), arr,
                                       out.ctypes.data_as(C.POINTER(C.c_float)), _stream(None)), "lfd_score")
        return out[:len(qs)]

    def get_superpixels(self, view: int) -> dict:
        S = int(self.S[view])
        off = np.zeros(S + 1, np.int32)
        h, w = self.view_hw[view] if getattr(self, "view_hw", None) else (self.H, self.W)
        pix = np.zeros(h * w, np.int32)
        stats = np.zeros((S, 8), np.float32)
        nb = np.zeros(MAX_NEIGHBOR_VIEWS, np.int32)
        self._check(self.lib.lfd_get_superpixels(self.h, view, off.ctypes.data, pix.ctypes.data, stats.ctypes.data,
                                                 nb.ctypes.data, _stream(None)), "lfd_get_superpixels")
        return dict(off=off, pix=pix, stats=stats, neighbours=nb[nb >= 0])


def terms_dict(rec: np.ndarray, nviews: int) -> dict:
    """Split one lfd_score record into named terms."""
    d = dict(E=float(rec[0]), Es=float(rec[1]), Ec=float(rec[2]), tssd=float(rec[3]))
    per = rec[TERMS_HEAD:TERMS_HEAD + nviews * TERMS_PER_VIEW].reshape(nviews, TERMS_PER_VIEW)
    d.update(S=per[:, 0], Vt=per[:, 1], O=per[:, 2], nvalid=per[:, 3], nx=per[:, 4], ny=per[:, 5])
    return d


class Server:
    """Frame server (lfd_server): rigs share one GPU by continuous batching
    over `max_slots` context+stream slots; later frames of a rig start warm
    from its previous planes."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, max_slots: int = 4):
        self.lib = load()
        self.h = C.c_void_p()
        st = self.lib.lfd_server_create(C.byref(self.h), device, hbm_budget, max_slots)
        if st != 0:
            raise LfdError(st, f"lfd_server_create: {self.lib.lfd_status_string(st).decode()}")
        self.device = device
        self._keep = {}

    def close(self):
        if self.h:
            self.lib.lfd_server_destroy(self.h)
            self.h = C.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != 0:
            raise LfdError(st, f"{what}: {self.lib.lfd_status_string(st).decode()}: "
                               f"{self.lib.lfd_server_last_error(self.h).decode()}")

    @staticmethod
    def now_ns() -> int:
        return int(load().lfd_server_now_ns())

    def configure(self, warm_iterations: int = 3, warm_iter_offset: int = 3, max_pending: int = 2):
        self._check(self.lib.lfd_server_configure(self.h, warm_iterations, warm_iter_offset, max_pending),
                    "lfd_server_configure")

    def submit(self, rig_id: int, views, labels, K, R, t, GW, GH, params: dict, planes_out=None, depth_out=None):
        """Queue a frame; returns the request id, or None when the rig already
        has its maximum of frames in flight (LFD_ERR_BUSY).  planes_out is a
        (S_total, 4) float32 cuda tensor, depth_out (V, H, W) float32, or None."""
        lf, keep = marshal_lightfield(views, labels, K, R, t, GW, GH)
        p = params_struct(params)
        V = len(K)
        pp = dd = None
        if planes_out is not None:
            S = [int(a) * int(b) for a, b in zip(np.broadcast_to(GW, V), np.broadcast_to(GH, V))]
            base = np.concatenate([[0], np.cumsum(S)[:-1]])
            pp = _ptr_array([planes_out.data_ptr() + int(b) * 16 for b in base])
        if depth_out is not None:
            dd = _ptr_array([depth_out[v].data_ptr() for v in range(V)])
        rid = C.c_uint64()
        st = self.lib.lfd_server_submit(self.h, rig_id, C.byref(lf), C.byref(p), pp, dd, C.byref(rid))
        if st == LFD_ERR_BUSY:
            return None
        self._check(st, "lfd_server_submit")
        self._keep[rid.value] = (lf, keep, p, pp, dd, planes_out, depth_out)
        return rid.value

    def poll(self, req_id: int, timeout_us: int = -1):
        """Result dict of a finished request, or None if still running after timeout_us."""
        r = Result()
        st = self.lib.lfd_server_poll(self.h, req_id, timeout_us, C.byref(r))
        if st == LFD_ERR_TIMEOUT:
            return None
        self._check(st, "lfd_server_poll")
        self._keep.pop(req_id, None)
        return dict(req_id=r.req_id, rig_id=r.rig_id, warm=r.warm, frame=r.frame, submit_ns=r.submit_ns,
                    done_ns=r.done_ns, status=r.status, slot=r.slot, start_ns=r.start_ns, batch=r.batch)

    def set_max_batch(self, n: int):
        self._check(self.lib.lfd_server_set_max_batch(self.h, int(n)), "lfd_server_set_max_batch")

    def stats(self) -> dict:
        b, f = C.c_int64(), C.c_int64()
        self._check(self.lib.lfd_server_stats(self.h, C.byref(b), C.byref(f)), "lfd_server_stats")
        return {"batches": b.value, "frames": f.value}

    def export_state(self, rig_id: int) -> torch.Tensor:
        n = C.c_int64()
        self._check(self.lib.lfd_server_export_state(self.h, rig_id, None, 0, C.byref(n)), "lfd_server_export_state")
        out = torch.zeros((n.value, 4), dtype=torch.float32)
        self._check(self.lib.lfd_server_export_state(self.h, rig_id, out.data_ptr(), n.value, C.byref(n)),
                    "lfd_server_export_state")
        return out

    def import_state(self, rig_id: int, planes: torch.Tensor):
        planes = planes.detach().to(torch.float32).cpu().contiguous()
        self._check(self.lib.lfd_server_import_state(self.h, rig_id, planes.data_ptr(), planes.shape[0]),
                    "lfd_server_import_state")
