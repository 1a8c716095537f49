"""ctypes binding of libaaag (include/aaag.h).

The functions below carry the C names and only marshal arguments: every step
of the renderer runs in the CUDA kernels of libaaag.so.  PyTorch provides the
device memory and the streams.  If the library is missing the import of this
module still works, but every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB_PATH

AAAG_OK = 0
AAAG_ERR_INVALID_ARG, AAAG_ERR_CAPACITY, AAAG_ERR_CUDA, AAAG_ERR_TIMEOUT, AAAG_ERR_UNSUPPORTED = 1, 2, 3, 4, 5
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CAPACITY", 3: "CUDA", 4: "TIMEOUT", 5: "UNSUPPORTED"}
AAAG_FLAG_NO_FILTER = 1
AAAG_FLAG_NO_CULL = 2
AAAG_FLAG_NO_RESORT = 4
AAAG_FLAG_KBUFFER = 8
AAAG_FLAG_EVAL_2D = 16
AAAG_STAGE_PREPROCESS, AAAG_STAGE_CULL, AAAG_STAGE_SORT, AAAG_STAGE_RENDER = 1, 2, 4, 8


class AaagError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class aaag_scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("reserved", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("vhat_train", C.c_void_p)]


class aaag_camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("bg", C.c_float * 3)]


class aaag_params(C.Structure):
    _fields_ = [("k", C.c_float), ("eps", C.c_float), ("flags", C.c_uint32), ("reserved", C.c_int32)]


class aaag_stats(C.Structure):
    _fields_ = [("n_gaussians", C.c_uint64), ("n_visible", C.c_uint64), ("n_pairs", C.c_uint64),
                ("pair_capacity", C.c_uint64), ("tiles_tested", C.c_uint64),
                ("evaluations", C.c_uint64), ("blended", C.c_uint64), ("misorders", C.c_uint64),
                ("extra_passes", C.c_uint64), ("replay_mismatch", C.c_uint64), ("capacity_overflow", C.c_uint32), ("timeout", C.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class aaag_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class aaag_workspace_view(C.Structure):
    _fields_ = [("records", C.c_void_p), ("aux", C.c_void_p), ("counts", C.c_void_p),
                ("offsets", C.c_void_p), ("keys_unsorted", C.c_void_p), ("vals_unsorted", C.c_void_p),
                ("keys_sorted", C.c_void_p), ("vals_sorted", C.c_void_p), ("tile_ranges", C.c_void_p),
                ("final_T", C.c_void_p), ("n_blended", C.c_void_p), ("tiles_x", C.c_int32),
                ("tiles_y", C.c_int32), ("tile_bits", C.c_int32), ("depth_shift", C.c_int32),
                ("depth_bits", C.c_int32)]


# (name, restype, argtypes) of every exported symbol
SIGNATURES = [
    ("aaag_workspace_bytes", C.c_size_t, [C.c_int64, C.c_int32, C.c_int32, C.c_int64]),
    ("aaag_workspace_init", C.c_int, [C.c_void_p, C.c_size_t, C.c_int64, C.c_int32, C.c_int32, C.c_int64,
                                      C.POINTER(C.c_void_p)]),
    ("aaag_workspace_destroy", None, [C.c_void_p]),
    ("aaag_workspace_get_view", C.c_int, [C.c_void_p, C.POINTER(aaag_workspace_view)]),
    ("aaag_preprocess", C.c_int, [C.POINTER(aaag_scene), C.POINTER(aaag_camera), C.POINTER(aaag_params),
                                  C.c_void_p, C.c_void_p]),
    ("aaag_cull", C.c_int, [C.c_void_p, C.c_void_p]),
    ("aaag_sort", C.c_int, [C.c_void_p, C.c_void_p]),
    ("aaag_render", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("aaag_render_frame", C.c_int, [C.POINTER(aaag_scene), C.POINTER(aaag_camera), C.POINTER(aaag_params),
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("aaag_render_backward", C.c_int, [C.POINTER(aaag_scene), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(aaag_grads), C.c_void_p]),
    ("aaag_render_batch", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.c_int32, C.c_void_p]),
    ("aaag_graph_create", C.c_int, [C.POINTER(aaag_scene), C.POINTER(aaag_camera), C.POINTER(aaag_params),
                                    C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    ("aaag_graph_launch", C.c_int, [C.c_void_p, C.POINTER(aaag_camera), C.c_void_p]),
    ("aaag_graph_destroy", None, [C.c_void_p]),
    ("aaag_selftest_wait_timeout", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    ("aaag_radix_sort_scratch_bytes", C.c_size_t, [C.c_int64]),
    ("aaag_radix_sort", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                  C.c_void_p, C.c_size_t, C.POINTER(C.c_int32), C.c_void_p]),
    ("aaag_radix_sort_static_capacity", C.c_int64, []),
    ("aaag_radix_sort_static", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    ("aaag_radix_sort_static_status", C.c_int, []),
    ("aaag_vhat_train", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("aaag_get_stats", C.c_int, [C.c_void_p, C.POINTER(aaag_stats), C.c_void_p]),
    ("aaag_last_error", C.c_char_p, []),
]

_lib = None


def lib():
    """The loaded libaaag.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, where):
    if status != AAAG_OK:
        raise AaagError(status, where, lib().aaag_last_error().decode())


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------

def aaag_workspace_bytes(n, width, height, pair_capacity):
    return int(lib().aaag_workspace_bytes(n, width, height, pair_capacity))


def aaag_workspace_init(dev_ptr, nbytes, n, width, height, pair_capacity):
    out = C.c_void_p()
    _check(lib().aaag_workspace_init(dev_ptr, nbytes, n, width, height, pair_capacity, C.byref(out)),
           "aaag_workspace_init")
    return out


def aaag_workspace_destroy(ws):
    lib().aaag_workspace_destroy(ws)


def aaag_workspace_get_view(ws):
    v = aaag_workspace_view()
    _check(lib().aaag_workspace_get_view(ws, C.byref(v)), "aaag_workspace_get_view")
    return v


def aaag_preprocess(scene, camera, params, ws, stream):
    _check(lib().aaag_preprocess(C.byref(scene), C.byref(camera),
                                 C.byref(params) if params is not None else None, ws, stream),
           "aaag_preprocess")


def aaag_cull(ws, stream):
    _check(lib().aaag_cull(ws, stream), "aaag_cull")


def aaag_sort(ws, stream):
    _check(lib().aaag_sort(ws, stream), "aaag_sort")


def aaag_render(ws, rgb_ptr, alpha_ptr, stream):
    _check(lib().aaag_render(ws, rgb_ptr, alpha_ptr, stream), "aaag_render")


def aaag_render_frame(scene, camera, params, ws, rgb_ptr, alpha_ptr, stream):
    _check(lib().aaag_render_frame(C.byref(scene), C.byref(camera),
                                   C.byref(params) if params is not None else None, ws,
                                   rgb_ptr, alpha_ptr, stream), "aaag_render_frame")


def aaag_render_backward(scene, ws, rgb_ptr, drgb_ptr, dalpha_ptr, grads, stream):
    _check(lib().aaag_render_backward(C.byref(scene), ws, rgb_ptr, drgb_ptr, dalpha_ptr, C.byref(grads), stream),
           "aaag_render_backward")


def aaag_render_batch(ws_handles, rgb_ptrs, alpha_ptrs, stream):
    n = len(ws_handles)
    W = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in ws_handles])
    R = (C.c_void_p * n)(*rgb_ptrs)
    A = (C.c_void_p * n)(*alpha_ptrs)
    _check(lib().aaag_render_batch(W, R, A, n, stream), "aaag_render_batch")


def aaag_graph_create(scene, camera, params, ws, stages, rgb_ptr, alpha_ptr, stream):
    out = C.c_void_p()
    _check(lib().aaag_graph_create(C.byref(scene), C.byref(camera),
                                   C.byref(params) if params is not None else None, ws, stages,
                                   rgb_ptr, alpha_ptr, stream, C.byref(out)), "aaag_graph_create")
    return out


def aaag_graph_launch(graph, camera, stream):
    _check(lib().aaag_graph_launch(graph, C.byref(camera), stream), "aaag_graph_launch")


def aaag_graph_destroy(graph):
    lib().aaag_graph_destroy(graph)


def aaag_selftest_wait_timeout(ws, which, stream):
    _check(lib().aaag_selftest_wait_timeout(ws, which, stream), "aaag_selftest_wait_timeout")


def aaag_radix_sort_scratch_bytes(n):
    return int(lib().aaag_radix_sort_scratch_bytes(n))


def aaag_radix_sort(keys, vals, keys_alt, vals_alt, n, key_bits, scratch, scratch_bytes, stream):
    alt = C.c_int32(0)
    _check(lib().aaag_radix_sort(keys, vals, keys_alt, vals_alt, n, key_bits, scratch, scratch_bytes,
                                 C.byref(alt), stream), "aaag_radix_sort")
    return int(alt.value)


def aaag_vhat_train(means_ptr, n, cams, out_ptr, stream):
    """cams: sequence of aaag_camera structs (host)."""
    arr = (aaag_camera * max(len(cams), 1))(*cams)
    _check(lib().aaag_vhat_train(means_ptr, n, C.cast(arr, C.c_void_p), len(cams), out_ptr, stream),
           "aaag_vhat_train")


def aaag_radix_sort_static_capacity():
    return int(lib().aaag_radix_sort_static_capacity())


def aaag_radix_sort_static(keys, vals, n, key_bits, stream):
    _check(lib().aaag_radix_sort_static(keys, vals, n, key_bits, stream), "aaag_radix_sort_static")


def aaag_radix_sort_static_status():
    """Status code of the last aaag_radix_sort_static on the current device
    (0 = OK, 4 = a bounded wait gave up); call after synchronising its stream."""
    return int(lib().aaag_radix_sort_static_status())


def aaag_get_stats(ws, stream, check=True):
    s = aaag_stats()
    st = lib().aaag_get_stats(ws, C.byref(s), stream)
    if check:
        _check(st, "aaag_get_stats")
    return s, st


def aaag_last_error():
    return lib().aaag_last_error().decode()


# ---------------------------------------------------------------------------
# torch-side marshalling helpers
# ---------------------------------------------------------------------------

def make_camera(cam) -> aaag_camera:
    """aaag_camera from a `scenes.Camera`."""
    c = aaag_camera()
    vm = np.asarray(cam.viewmat, dtype=np.float32).reshape(16)
    for i in range(16):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = cam.znear
    for i in range(3):
        c.bg[i] = cam.bg[i]
    return c


def make_params(k=0.3, eps=1e-3, flags=0) -> aaag_params:
    return aaag_params(k, eps, flags, 0)


class DeviceScene:
    """Scene arrays resident on the GPU (float32, contiguous)."""

    def __init__(self, scene, device="cuda"):
        import torch
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)
        self.means = t(scene.means)
        self.log_scales = t(scene.log_scales)
        self.quats = t(scene.quats)
        self.opacity_logits = t(scene.opacity_logits)
        self.sh = t(scene.sh)
        self.vhat_train = t(scene.vhat_train)
        self.sh_degree = int(scene.sh_degree)
        self.n = int(scene.n)

    def struct(self) -> aaag_scene:
        return aaag_scene(self.n, self.sh_degree, 0, self.means.data_ptr(), self.log_scales.data_ptr(),
                          self.quats.data_ptr(), self.opacity_logits.data_ptr(), self.sh.data_ptr(),
                          self.vhat_train.data_ptr())


class Workspace:
    """Device workspace for n Gaussians, one image size and a pair capacity."""

    def __init__(self, n, width, height, pair_capacity, device="cuda"):
        import torch
        self.n, self.width, self.height, self.capacity = int(n), int(width), int(height), int(pair_capacity)
        self.nbytes = aaag_workspace_bytes(self.n, self.width, self.height, self.capacity)
        self.buffer = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        base = self.buffer.data_ptr()
        self.ptr = base + (-base) % 256
        self.handle = aaag_workspace_init(self.ptr, self.nbytes, self.n, self.width, self.height, self.capacity)

    def view(self):
        return aaag_workspace_get_view(self.handle)

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                aaag_workspace_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def render(dscene: DeviceScene, cam, ws: Workspace, params=None, rgb=None, alpha=None, stream=None):
    """Render one frame into (rgb [3,H,W], alpha [H,W]) float32 CUDA tensors."""
    import torch
    if rgb is None:
        rgb = torch.empty(3, cam.height, cam.width, dtype=torch.float32, device=dscene.means.device)
    if alpha is None:
        alpha = torch.empty(cam.height, cam.width, dtype=torch.float32, device=dscene.means.device)
    aaag_render_frame(dscene.struct(), make_camera(cam), params if params is not None else make_params(),
                      ws.handle, rgb.data_ptr(), alpha.data_ptr(),
                      stream if stream is not None else current_stream())
    return rgb, alpha


def stats(ws: Workspace, stream=None, check=True):
    s, st = aaag_get_stats(ws.handle, stream if stream is not None else current_stream(), check)
    d = s.as_dict()
    d["status"] = STATUS_NAMES.get(st, st)
    return d
