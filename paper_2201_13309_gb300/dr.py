"""Python binding of libdr (include/dr.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python
values into the C structs, passes torch tensors' device pointers and CUDA
stream handles through, and turns status codes into exceptions.  There is no
fallback: if libdr.so is missing or has no GPU to run on, calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DR_LIBRARY selects another build of the same library (the bounds-checked
# test build, libdr_checked.so); the default is the in-tree libdr.so
LIB_PATH = os.environ.get("DR_LIBRARY") or os.path.join(HERE, "libdr.so")

DR_OK = 0
STATUS = {0: "DR_OK", 1: "DR_ERR_INVALID_ARG", 2: "DR_ERR_GEOMETRY",
          3: "DR_ERR_NONMONOTONIC", 4: "DR_ERR_OOM", 5: "DR_ERR_BUDGET",
          6: "DR_ERR_CUDA", 7: "DR_ERR_TIMEOUT", 8: "DR_ERR_UNSUPPORTED"}
EDGES = {"leading": 0, "trailing": 1, "both": 2}
OUT_DTYPES = {"f32": 0, "bf16": 1}
GEOM_PRECISIONS = {"fp32": 0, "fp64": 1}
DEPTH_FORMS = {"auto": 0, "exact": 1, "series": 2, "poly": 3}
KERNELS = {0: "rows", 1: "pixels", 2: "intervals"}

# every symbol include/dr.h declares (checked by the CPU tests)
EXPORTS = ("dr_plan", "dr_plan_destroy", "dr_plan_get_info", "dr_plan_device_bytes",
           "dr_reconstruct", "dr_reconstruct_host", "dr_image_differences",
           "dr_plan_depths", "dr_plan_check", "dr_selftest_wait_timeout",
           "dr_status_string", "dr_last_error",
           "dr_version", "dr_reconstruct_rows_static", "dr_batch_create", "dr_batch_launch",
           "dr_batch_check", "dr_batch_get_info", "dr_batch_destroy", "dr_batch_reconstruct",
           "dr_server_create",
           "dr_server_submit", "dr_server_poll", "dr_server_wait", "dr_server_fetch",
           "dr_server_fetch_into", "dr_server_release", "dr_server_get_stats",
           "dr_server_destroy", "dr_reconstruct_streamed", "dr_pixel_activity",
           "dr_select_scratch_bytes", "dr_select_pixels", "dr_reconstruct_selected")
REQ_STATES = {0: "queued", 1: "uploading", 2: "running", 3: "done", 4: "failed"}

_d3 = ctypes.c_double * 3


class Geometry(ctypes.Structure):
    _fields_ = [("beam_origin", _d3), ("beam_dir", _d3), ("det_origin", _d3),
                ("row_step", _d3), ("col_step", _d3), ("rows", ctypes.c_int32),
                ("cols", ctypes.c_int32), ("wire_axis", _d3),
                ("wire_radius", ctypes.c_double), ("edge", ctypes.c_int32)]


class PlanOptions(ctypes.Structure):
    _fields_ = [("out_dtype", ctypes.c_int32), ("geom_precision", ctypes.c_int32),
                ("tile_cols", ctypes.c_int32), ("bin_groups", ctypes.c_int32),
                ("force_pixels", ctypes.c_int32), ("force_intervals", ctypes.c_int32),
                ("depth_form", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "rows", "cols", "K", "B", "kernel", "tile_cols", "pixels_per_thread",
        "bin_groups", "threads", "smem_bytes", "tma_chunk", "tma_chunks", "out_dtype",
        "geom_precision", "edge", "reversed", "fixed_shift", "row_tables", "parts")] + [
        ("depth_min", ctypes.c_double), ("depth_max", ctypes.c_double),
        ("min_step", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
        ("bytes_per_call", ctypes.c_double), ("max_step", ctypes.c_double),
        ("depth_err", ctypes.c_double), ("depth_form", ctypes.c_int32),
        ("one_step_per_bin", ctypes.c_int32), ("checked_groups", ctypes.c_int64)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_}
        d["kernel"] = KERNELS.get(d["kernel"], d["kernel"])
        return d


class Job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_images", ctypes.c_void_p),
                ("d_out", ctypes.c_void_p)]


class BatchOptions(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("max_tile_cols", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("scans", ctypes.c_int32), ("items", ctypes.c_int64), ("grid", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("device_bytes", ctypes.c_size_t)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("slots", ctypes.c_int32),
                ("plan_cache", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_double), ("admitted", ctypes.c_double),
                ("planned", ctypes.c_double), ("uploaded", ctypes.c_double),
                ("done", ctypes.c_double), ("issued", ctypes.c_double),
                ("copy", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("queued", "in_flight", "admitted", "completed",
                                               "failed", "plans_built", "plans_cached")] + [
        ("arena_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t)]


class DrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def lib():
    """Load libdr.so (built in-tree by __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, I32, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
            sig = {
                "dr_plan": ([ctypes.POINTER(Geometry), P, I32, P, I32,
                             ctypes.POINTER(PlanOptions), ctypes.POINTER(P)], I32),
                "dr_plan_destroy": ([P], None),
                "dr_plan_get_info": ([P, ctypes.POINTER(PlanInfo)], I32),
                "dr_plan_device_bytes": ([P], SZ),
                "dr_reconstruct": ([P, P, P, P], I32),
                "dr_reconstruct_host": ([P, P, P, P, P, P], I32),
                "dr_image_differences": ([P, I32, I32, I32, P, P], I32),
                "dr_plan_depths": ([P, I32, I32, P, P], I32),
                "dr_plan_check": ([P], I32),
                "dr_selftest_wait_timeout": ([P, ctypes.c_double, P], I32),
                "dr_status_string": ([I32], ctypes.c_char_p),
                "dr_last_error": ([], ctypes.c_char_p),
                "dr_version": ([], ctypes.c_char_p),
                "dr_reconstruct_rows_static": ([ctypes.POINTER(Geometry), P, I32, P, I32, P, P,
                                                P, P], I32),
                "dr_batch_create": ([ctypes.POINTER(Job), I32, ctypes.POINTER(BatchOptions),
                                     ctypes.POINTER(P)], I32),
                "dr_batch_launch": ([P, P], I32),
                "dr_batch_check": ([P], I32),
                "dr_batch_get_info": ([P, ctypes.POINTER(BatchInfo)], I32),
                "dr_batch_destroy": ([P], None),
                "dr_batch_reconstruct": ([ctypes.POINTER(Job), I32, ctypes.POINTER(BatchOptions),
                                          P], I32),
                "dr_server_create": ([ctypes.POINTER(ServerOptions), ctypes.POINTER(P)], I32),
                "dr_server_submit": ([P, ctypes.POINTER(Geometry), P, I32, P, I32, P,
                                      ctypes.POINTER(ctypes.c_uint64)], I32),
                "dr_server_poll": ([P, ctypes.c_uint64, ctypes.POINTER(I32)], I32),
                "dr_server_wait": ([P, ctypes.c_uint64, ctypes.c_double], I32),
                "dr_server_fetch": ([P, ctypes.c_uint64, ctypes.POINTER(P),
                                     ctypes.POINTER(RequestTimes)], I32),
                "dr_server_fetch_into": ([P, ctypes.c_uint64, P, SZ, P], I32),
                "dr_server_release": ([P, ctypes.c_uint64], I32),
                "dr_server_get_stats": ([P, ctypes.POINTER(ServerStats)], I32),
                "dr_server_destroy": ([P], None),
                "dr_reconstruct_streamed": ([P, P, P, P, SZ, I32, P], I32),
                "dr_pixel_activity": ([P, I32, I32, I32, P, P], I32),
                "dr_select_scratch_bytes": ([ctypes.c_int64], SZ),
                "dr_select_pixels": ([P, ctypes.c_int64, ctypes.c_float, P, P, P, SZ, P], I32),
                "dr_reconstruct_selected": ([P, P, P, I32, P, P], I32),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def check(status):
    if status != DR_OK:
        raise DrError(status, lib().dr_last_error().decode())


def geometry_struct(geom, edge="leading"):
    g = Geometry()
    for key in ("beam_origin", "beam_dir", "det_origin", "row_step", "col_step",
                "wire_axis"):
        setattr(g, key, _d3(*[float(v) for v in geom[key]]))
    g.rows = int(geom["rows"])
    g.cols = int(geom["cols"])
    g.wire_radius = float(geom["wire_radius"])
    g.edge = EDGES[edge] if isinstance(edge, str) else int(edge)
    return g


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _require(t, what, shape=None, dtype=None, int16=False, cuda=True):
    """Checks a tensor handed to the C ABI by address (the library cannot
    see buffer sizes or types): its shape, element type, contiguity and
    whether it lives in device or host memory.  ValueError before any call."""
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} {tuple(t.shape)} != {tuple(shape)}")
    if int16 and (t.element_size() != 2 or t.is_floating_point() or t.is_complex()):
        raise ValueError(f"{what} must hold 16-bit integers, got {t.dtype}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{what} dtype {t.dtype} != {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if bool(t.is_cuda) != cuda:
        raise ValueError(f"{what} must be in {'device' if cuda else 'host'} memory")


class Plan:
    """A reconstruction plan (dr_plan): geometry, wire path and bin edges.

    geom: dict with beam_origin, beam_dir, det_origin, row_step, col_step,
    rows, cols, wire_axis, wire_radius (mm); wires [K, 3]; edges [B + 1]
    (depth, mm, strictly increasing).  edge: "leading", "trailing" or
    "both"; out_dtype "f32" / "bf16"; geom_precision "fp32" / "fp64";
    tile_cols / bin_groups: launch shape (0 = default); force_pixels /
    force_intervals: use the per-pixel or the interval kernel instead of the
    one the plan picks (info()["kernel"] tells which); depth_form: "auto",
    or the most elaborate form of the FP32 depth remainder the plan may use
    ("exact", "series", "poly"; info()["depth_form"] tells which it took).
    """

    def __init__(self, geom, wires, edges, edge="leading", out_dtype="f32",
                 geom_precision="fp32", tile_cols=0, bin_groups=0, force_pixels=False,
                 force_intervals=False, depth_form="auto"):
        L = lib()
        self._wires = np.ascontiguousarray(wires, dtype=np.float64)
        self._edges = np.ascontiguousarray(edges, dtype=np.float64)
        self.geom = dict(geom)
        self.edge = edge
        self.out_dtype = out_dtype
        g = geometry_struct(geom, edge)
        o = PlanOptions()
        o.out_dtype = OUT_DTYPES[out_dtype]
        o.geom_precision = GEOM_PRECISIONS[geom_precision]
        o.tile_cols = int(tile_cols)
        o.bin_groups = int(bin_groups)
        o.force_pixels = 1 if force_pixels else 0
        o.force_intervals = 1 if force_intervals else 0
        o.depth_form = DEPTH_FORMS[depth_form]
        h = ctypes.c_void_p()
        check(L.dr_plan(ctypes.byref(g), self._wires.ctypes.data_as(ctypes.c_void_p),
                        self._wires.shape[0], self._edges.ctypes.data_as(ctypes.c_void_p),
                        self._edges.shape[0] - 1, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.K = int(self._wires.shape[0])
        self.B = int(self._edges.shape[0] - 1)
        self.rows = int(geom["rows"])
        self.cols = int(geom["cols"])

    @property
    def handle(self):
        return self._h

    def info(self):
        i = PlanInfo()
        check(lib().dr_plan_get_info(self._h, ctypes.byref(i)))
        return i.as_dict()

    def out_torch_dtype(self):
        import torch
        return torch.bfloat16 if self.out_dtype == "bf16" else torch.float32

    def empty_output(self, device="cuda"):
        import torch
        return torch.empty((self.B, self.rows, self.cols), dtype=self.out_torch_dtype(),
                           device=device)

    def reconstruct(self, images, out=None, stream=None):
        """images: CUDA tensor [K, rows, cols] of uint16 bits (int16 or uint16
        dtype); out: CUDA tensor [B, rows, cols] (allocated if None)."""
        if out is None:
            out = self.empty_output(images.device)
        self._check_shapes(images, out)
        check(lib().dr_reconstruct(self._h, _dptr(images), _dptr(out),
                                   ctypes.c_void_p(_stream_handle(stream))))
        return out

    def reconstruct_host(self, h_images, h_out, d_images, d_out, stream=None):
        """End to end: pinned host images -> device -> reconstruct -> host."""
        self._check_host(h_images, h_out)
        self._check_shapes(d_images, d_out)
        check(lib().dr_reconstruct_host(self._h, _dptr(h_images), _dptr(h_out),
                                        _dptr(d_images), _dptr(d_out),
                                        ctypes.c_void_p(_stream_handle(stream))))
        return h_out

    def reconstruct_streamed(self, h_images, h_out, workspace, slab_rows=0, stream=None):
        """Out-of-core form: host images -> row slabs through a device
        workspace (a CUDA tensor; three slab buffers) -> host output."""
        self._check_host(h_images, h_out)
        _require(workspace, "workspace")
        check(lib().dr_reconstruct_streamed(
            self._h, _dptr(h_images), _dptr(h_out), _dptr(workspace),
            workspace.numel() * workspace.element_size(), int(slab_rows),
            ctypes.c_void_p(_stream_handle(stream))))
        return h_out

    def reconstruct_selected(self, images, index, n=None, out=None, stream=None):
        """Bins of the listed pixels only: out [B, n], out[:, i] = bin values
        of pixel index[i] (row-major; int32, each in [0, rows * cols)).  n
        defaults to len(index)."""
        import torch
        n = int(index.numel() if n is None else n)
        if out is None:
            out = torch.empty((self.B, n), dtype=self.out_torch_dtype(), device=images.device)
        _require(images, "images", (self.K, self.rows, self.cols), int16=True)
        _require(index, "index", dtype=torch.int32)
        if index.dim() != 1 or not 0 <= n <= index.numel():
            raise ValueError(f"index must be one-dimensional with at least n = {n} entries")
        _require(out, "out", dtype=self.out_torch_dtype())
        if out.dim() != 2 or out.shape[0] != self.B or (n > 0 and out.shape[1] != n):
            raise ValueError(f"out {tuple(out.shape)} != {(self.B, n)}")
        check(lib().dr_reconstruct_selected(self._h, _dptr(images), _dptr(index), n,
                                            _dptr(out), ctypes.c_void_p(_stream_handle(stream))))
        return out

    def depths(self, r0=0, nrows=None, stream=None):
        """The GPU's depths d_k (mm) for rows r0..: CUDA float64 [nrows, cols, K]."""
        import torch
        nrows = self.rows - r0 if nrows is None else nrows
        d = torch.empty((nrows, self.cols, self.K), dtype=torch.float64, device="cuda")
        check(lib().dr_plan_depths(self._h, r0, nrows, _dptr(d),
                                   ctypes.c_void_p(_stream_handle(stream))))
        return d

    def check_device(self):
        check(lib().dr_plan_check(self._h))

    def _check_shapes(self, images, out):
        _require(images, "images", (self.K, self.rows, self.cols), int16=True)
        _require(out, "out", (self.B, self.rows, self.cols), dtype=self.out_torch_dtype())

    def _check_host(self, h_images, h_out):
        _require(h_images, "h_images", (self.K, self.rows, self.cols), int16=True, cuda=False)
        _require(h_out, "h_out", (self.B, self.rows, self.cols), dtype=self.out_torch_dtype(),
                 cuda=False)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().dr_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _jobs_array(jobs):
    arr = (Job * len(jobs))()
    for i, (plan, images, out) in enumerate(jobs):
        plan._check_shapes(images, out)
        arr[i].plan = plan.handle
        arr[i].d_images = images.data_ptr()
        arr[i].d_out = out.data_ptr()
    return arr


def _batch_options(ctas_per_sm=0, max_tile_cols=0, threads=0):
    o = BatchOptions()
    o.ctas_per_sm = int(ctas_per_sm)
    o.max_tile_cols = int(max_tile_cols)
    o.threads = int(threads)
    return o


def batch_reconstruct(jobs, stream=None, **options):
    """dr_batch_reconstruct: the (plan, images, out) jobs in one persistent
    launch, built, run, waited for and released in one call."""
    arr = _jobs_array(jobs)
    check(lib().dr_batch_reconstruct(arr, len(jobs), ctypes.byref(_batch_options(**options)),
                                     ctypes.c_void_p(_stream_handle(stream))))


class Batch:
    """dr_batch: several (plan, images, out) jobs reconstructed by one
    persistent launch replayed from a CUDA graph.  The tensors are bound at
    creation and must stay alive (and in place) while the batch exists."""

    def __init__(self, jobs, ctas_per_sm=0, max_tile_cols=0, threads=0):
        self._keep = list(jobs)
        self.ctas_per_sm = ctas_per_sm
        arr = _jobs_array(jobs)
        o = _batch_options(ctas_per_sm, max_tile_cols, threads)
        h = ctypes.c_void_p()
        check(lib().dr_batch_create(arr, len(jobs), ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        check(lib().dr_batch_launch(self._h, ctypes.c_void_p(_stream_handle(stream))))

    def check_device(self):
        check(lib().dr_batch_check(self._h))

    def info(self):
        i = BatchInfo()
        check(lib().dr_batch_get_info(self._h, ctypes.byref(i)))
        return {n: getattr(i, n) for n, _ in i._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().dr_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """dr_server: continuous admission of reconstruction requests against a
    device-memory budget; results stay on the device until released."""

    def __init__(self, budget_bytes, slots=0, plan_cache=0):
        o = ServerOptions()
        o.budget_bytes = int(budget_bytes)
        o.slots = int(slots)
        o.plan_cache = int(plan_cache)
        h = ctypes.c_void_p()
        check(lib().dr_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._pinned = {}

    def submit(self, geom, wires, edges, h_images, edge="leading"):
        """h_images: host (pinned) 16-bit tensor [K, rows, cols]; kept alive
        by the server object until the request is released."""
        w = np.ascontiguousarray(wires, dtype=np.float64)
        e = np.ascontiguousarray(edges, dtype=np.float64)
        if w.ndim != 2 or w.shape[1] != 3 or e.ndim != 1 or e.shape[0] < 2:
            raise ValueError(f"wires must be [K, 3] and edges [B + 1], got {w.shape}, {e.shape}")
        _require(h_images, "h_images", (w.shape[0], int(geom["rows"]), int(geom["cols"])),
                 int16=True, cuda=False)
        g = geometry_struct(geom, edge)
        rid = ctypes.c_uint64()
        check(lib().dr_server_submit(self._h, ctypes.byref(g), w.ctypes.data_as(ctypes.c_void_p),
                                     w.shape[0], e.ctypes.data_as(ctypes.c_void_p),
                                     e.shape[0] - 1, _dptr(h_images), ctypes.byref(rid)))
        self._pinned[rid.value] = h_images
        return rid.value

    def poll(self, rid):
        st = ctypes.c_int32()
        check(lib().dr_server_poll(self._h, rid, ctypes.byref(st)))
        return REQ_STATES[st.value]

    def wait(self, rid, timeout=600.0):
        check(lib().dr_server_wait(self._h, rid, float(timeout)))

    def fetch(self, rid):
        """(device address of the output, timestamps in s since creation)."""
        p = ctypes.c_void_p()
        t = RequestTimes()
        check(lib().dr_server_fetch(self._h, rid, ctypes.byref(p), ctypes.byref(t)))
        return p.value, {n: getattr(t, n) for n, _ in t._fields_}

    def fetch_into(self, rid, dst, stream=None):
        check(lib().dr_server_fetch_into(self._h, rid, _dptr(dst),
                                         dst.numel() * dst.element_size(),
                                         ctypes.c_void_p(_stream_handle(stream))))
        return dst

    def release(self, rid):
        check(lib().dr_server_release(self._h, rid))
        self._pinned.pop(rid, None)

    def stats(self):
        s = ServerStats()
        check(lib().dr_server_get_stats(self._h, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().dr_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._pinned.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def image_differences(images, stream=None):
    """int32 [K-1, rows, cols]: exact I_k - I_{k+1} as the kernels form it."""
    import torch
    K, H, W = images.shape
    _require(images, "images", int16=True)
    d = torch.empty((max(K - 1, 0), H, W), dtype=torch.int32, device=images.device)
    check(lib().dr_image_differences(_dptr(images), K, H, W, _dptr(d),
                                     ctypes.c_void_p(_stream_handle(stream))))
    return d


def reconstruct_rows_static(geom, wires, edges, images, out, status=None, edge="leading",
                            stream=None):
    """dr_reconstruct_rows_static: the rows kernel with no allocation at all.

    images: CUDA [K, rows, cols] 16-bit; out: CUDA float32 [B, rows, cols]
    (caller-allocated); status: optional CUDA int32 tensor of one element
    (with None, a device-side error code is not reported).  The C entry
    point cannot see buffer sizes, so every shape, type, layout and device is
    checked here before the call (ValueError).
    """
    import torch
    w = np.ascontiguousarray(wires, dtype=np.float64)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    if w.ndim != 2 or w.shape[1] != 3:
        raise ValueError(f"wires must be [K, 3], got {w.shape}")
    if e.ndim != 1 or e.shape[0] < 2:
        raise ValueError(f"edges must be [B + 1] with B >= 1, got {e.shape}")
    K, B = int(w.shape[0]), int(e.shape[0] - 1)
    H, W = int(geom["rows"]), int(geom["cols"])
    if H * W > 0:
        if images is None or out is None:
            raise ValueError("images and out are required for a non-empty ROI")
        if tuple(images.shape) != (K, H, W):
            raise ValueError(f"images {tuple(images.shape)} != {(K, H, W)}")
        if images.element_size() != 2 or images.is_floating_point() or not images.is_contiguous():
            raise ValueError("images must be a contiguous 16-bit integer tensor")
        if tuple(out.shape) != (B, H, W):
            raise ValueError(f"out {tuple(out.shape)} != {(B, H, W)}")
        if out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 tensor")
    if status is not None and (status.dtype != torch.int32 or status.numel() != 1):
        raise ValueError("status must be a one-element int32 tensor")
    on_device = [status] + ([images, out] if H * W > 0 else [])
    for t in on_device:
        if t is not None and (not t.is_cuda or t.device.index != torch.cuda.current_device()):
            raise ValueError("images, out and status must be on the current CUDA device")
    g = geometry_struct(geom, edge)
    check(lib().dr_reconstruct_rows_static(
        ctypes.byref(g), w.ctypes.data_as(ctypes.c_void_p), w.shape[0],
        e.ctypes.data_as(ctypes.c_void_p), e.shape[0] - 1,
        None if images is None else _dptr(images), None if out is None else _dptr(out),
        None if status is None else _dptr(status), ctypes.c_void_p(_stream_handle(stream))))
    return out


def pixel_activity(images, stream=None):
    """float32 [rows, cols]: sum_k |I_k - I_{k+1}| per pixel (exact)."""
    import torch
    K, H, W = images.shape
    _require(images, "images", int16=True)
    act = torch.empty((H, W), dtype=torch.float32, device=images.device)
    check(lib().dr_pixel_activity(_dptr(images), K, H, W, _dptr(act),
                                  ctypes.c_void_p(_stream_handle(stream))))
    return act


def select_pixels(activity, threshold, stream=None):
    """(int32 index tensor of the pixels with activity >= threshold, in
    increasing row-major order; their count)."""
    import torch
    _require(activity, "activity", dtype=torch.float32)
    n = activity.numel()
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=activity.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=activity.device)
    scratch = torch.empty(int(lib().dr_select_scratch_bytes(n)), dtype=torch.uint8,
                          device=activity.device)
    check(lib().dr_select_pixels(_dptr(activity), n, float(threshold), _dptr(idx), _dptr(cnt),
                                 _dptr(scratch), scratch.numel(),
                                 ctypes.c_void_p(_stream_handle(stream))))
    count = int(cnt.item())
    return idx[:count], count


def version():
    return lib().dr_version().decode()


def selftest_wait_timeout(wait_ms=20.0, stream=None):
    """dr_selftest_wait_timeout: run the bounded-wait failure path once.
    Returns (status code, the device status word)."""
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib().dr_selftest_wait_timeout(_dptr(status), float(wait_ms),
                                         ctypes.c_void_p(_stream_handle(stream)))
    return st, int(status.item())
