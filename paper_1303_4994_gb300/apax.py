"""Python binding of the C ABI in include/apax.h (argument marshalling only).

Every step of the codec runs in the sm_103a kernels of libapax_gb300.so;
torch supplies device memory and streams.  The library must be built
(``paper_1303_4994_gb300.build.build()``); without it every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libapax_gb300.so")

I8, I16, I32, F32, F64 = 1, 2, 3, 4, 5
FIXED_RATE, FIXED_QUALITY = 0, 1
TORCH_CODE = {torch.int8: I8, torch.int16: I16, torch.int32: I32, torch.float32: F32,
              torch.float64: F64}
CODE_TORCH = {v: k for k, v in TORCH_CODE.items()}
ELEM_SIZE = {I8: 1, I16: 2, I32: 4, F32: 4, F64: 8}

STATUS = {0: "ok", -1: "invalid argument", -2: "block size", -3: "dtype", -4: "rate",
          -5: "capacity", -6: "too large", -7: "cuda", -8: "non-finite", -9: "corrupt",
          -10: "timeout"}
DEFAULT_CANDIDATES = tuple(256 * i for i in range(16))


class ApaxError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_uint32), ("mode", ctypes.c_int32),
                ("rate_num", ctypes.c_uint32), ("rate_den", ctypes.c_uint32),
                ("atten_code", ctypes.c_uint32), ("search", ctypes.c_uint32),
                ("format", ctypes.c_uint32)]


class Point(ctypes.Structure):
    _fields_ = [("code", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("bytes", ctypes.c_uint64),
                ("sx", ctypes.c_double), ("sy", ctypes.c_double), ("sxx", ctypes.c_double),
                ("sxy", ctypes.c_double), ("syy", ctypes.c_double), ("sdd", ctypes.c_double),
                ("r", ctypes.c_double)]


class Summary(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("recommended", ctypes.c_int32),
                ("recommended_code", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("n", ctypes.c_uint64)]


class EncodeJob(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("reserved0", ctypes.c_uint32),
                ("n", ctypes.c_uint64), ("p", Params), ("code_dev", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("out_capacity", ctypes.c_uint64),
                ("res", ctypes.c_void_p)]


class DecodeJob(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("in_bytes", ctypes.c_uint64), ("y", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("block_size", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("res", ctypes.c_void_p)]


class ProfileJob(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("block_size", ctypes.c_uint32),
                ("n", ctypes.c_uint64), ("candidates", ctypes.c_void_p), ("ncand", ctypes.c_int32),
                ("format", ctypes.c_uint32), ("target", ctypes.c_double),
                ("points", ctypes.c_void_p), ("summary", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_uint64),
                ("slots", ctypes.c_uint32), ("max_batch", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("op", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("n", ctypes.c_uint64), ("p", Params), ("in_", ctypes.c_void_p),
                ("in_bytes", ctypes.c_uint64), ("out", ctypes.c_void_p),
                ("out_capacity", ctypes.c_uint64), ("t_arrival", ctypes.c_double)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("op", ctypes.c_int32), ("status", ctypes.c_int32),
                ("bytes", ctypes.c_uint64), ("out", ctypes.c_void_p),
                ("t_arrival", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("queued", "inflight", "busy_slots", "arena_used",
                                                "arena_peak", "steps", "admitted", "completed",
                                                "undelivered")]


class Quality(ctypes.Structure):
    _fields_ = [("s2r_ratio", ctypes.c_double), ("n", ctypes.c_uint64), ("L", ctypes.c_uint32),
                ("segments", ctypes.c_uint32), ("peak_x", ctypes.c_double),
                ("floor_x", ctypes.c_double), ("peak_y", ctypes.c_double),
                ("floor_y", ctypes.c_double), ("peak_d", ctypes.c_double),
                ("floor_d", ctypes.c_double), ("mean_d_db", ctypes.c_double)]


QUALITY_DB = ("s2r_2sigma", "peak_x", "floor_x", "peak_y", "floor_y", "peak_d", "floor_d",
              "mean_d", "dr", "srr", "fft_s2r_margin")


class Shard(ctypes.Structure):
    _fields_ = [("container", ctypes.c_void_p), ("bytes", ctypes.c_uint64),
                ("block_begin", ctypes.c_uint64), ("block_end", ctypes.c_uint64)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32)]


POINT_BYTES = ctypes.sizeof(Point)
SUMMARY_BYTES = ctypes.sizeof(Summary)
RESULT_BYTES = 16

_lib = None

EXPORTS = ("apax_encoded_size", "apax_workspace_size", "apax_encode", "apax_encode_recommended",
           "apax_copy_container",
           "apax_decode_workspace_size", "apax_decode", "apax_decode_blocks",
           "apax_profile_workspace_size", "apax_profile", "apax_profile_format",
           "apax_profile_from_host",
           "apax_derived_metrics",
           "apax_encode_test_stall", "apax_status_string", "apax_build_info",
           "apax_encode_noalloc", "apax_batch_encode_workspace_size", "apax_batch_encode_create",
           "apax_batch_run", "apax_batch_get_config", "apax_batch_set_config", "apax_batch_tune",
           "apax_batch_tiles", "apax_batch_destroy", "apax_batch_decode_workspace_size",
           "apax_batch_decode_create", "apax_batch_profile_workspace_size",
           "apax_batch_profile_create", "apax_server_create", "apax_server_submit",
           "apax_server_poll", "apax_server_release", "apax_server_stats", "apax_server_destroy",
           "apax_shard_elements", "apax_encode_shard", "apax_shard_rebase", "apax_merge_shards",
           "apax_quality_workspace_size", "apax_quality_metrics", "apax_quality_db")
OP_ENCODE, OP_DECODE = 0, 1
NOALLOC_SCRATCH_BYTES = 256 << 10


def lib():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1303_4994_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, i32, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
        pP, p64 = ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_uint64)
        L.apax_encoded_size.argtypes = [i32, u64, pP, p64]
        L.apax_workspace_size.argtypes = [i32, u64, pP, p64]
        L.apax_encode.argtypes = [vp, i32, u64, pP, vp, u64, vp, u64, vp, vp]
        L.apax_encode_recommended.argtypes = [vp, i32, u64, pP, vp, vp, u64, vp, u64, vp, vp]
        L.apax_copy_container.argtypes = [vp, vp, vp, u64, vp]
        L.apax_decode_workspace_size.argtypes = []
        L.apax_decode_workspace_size.restype = u64
        L.apax_decode.argtypes = [vp, u64, vp, i32, u64, vp, u64, vp, vp]
        L.apax_decode_blocks.argtypes = [vp, u64, u64, u64, vp, i32, u64, vp, u64, vp, vp]
        L.apax_profile_workspace_size.argtypes = [i32, u64, u32, i32, p64]
        L.apax_profile.argtypes = [vp, i32, u64, u32, vp, i32, ctypes.c_double, vp, u64, vp, vp,
                                   vp]
        L.apax_profile_format.argtypes = [vp, i32, u64, u32, u32, vp, i32, ctypes.c_double, vp,
                                          u64, vp, vp, vp]
        L.apax_profile_from_host.argtypes = [vp, vp, i32, u64, u32, vp, i32, ctypes.c_double, i32,
                                             vp, u64, vp, vp, vp, vp]
        L.apax_derived_metrics.argtypes = [ctypes.POINTER(Point), u64, vp]
        L.apax_derived_metrics.restype = None
        L.apax_encode_test_stall.argtypes = [vp, i32, u64, pP, vp, u64, vp, u64, vp,
                                             ctypes.c_int64, ctypes.c_int64, vp]
        L.apax_encode_noalloc.argtypes = [vp, i32, u64, pP, vp, u64, vp, vp]
        pJ, pC = ctypes.POINTER(EncodeJob), ctypes.POINTER(BatchConfig)
        L.apax_batch_encode_workspace_size.argtypes = [pJ, i32, p64]
        L.apax_batch_encode_create.argtypes = [pJ, i32, vp, u64, ctypes.POINTER(vp)]
        pD, pPJ = ctypes.POINTER(DecodeJob), ctypes.POINTER(ProfileJob)
        L.apax_batch_profile_workspace_size.argtypes = [pPJ, i32, p64]
        L.apax_batch_profile_create.argtypes = [pPJ, i32, vp, u64, ctypes.POINTER(vp)]
        L.apax_batch_decode_workspace_size.argtypes = [pD, i32, p64]
        L.apax_batch_decode_create.argtypes = [pD, i32, vp, u64, ctypes.POINTER(vp)]
        L.apax_batch_run.argtypes = [vp, vp]
        L.apax_batch_get_config.argtypes = [vp, pC]
        L.apax_batch_set_config.argtypes = [vp, pC]
        L.apax_batch_tune.argtypes = [vp, i32, vp]
        L.apax_batch_tiles.argtypes = [vp]
        L.apax_batch_tiles.restype = u64
        L.apax_batch_destroy.argtypes = [vp]
        L.apax_batch_destroy.restype = None
        L.apax_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        L.apax_server_submit.argtypes = [vp, ctypes.POINTER(Request)]
        L.apax_server_poll.argtypes = [vp, ctypes.POINTER(Completion), i32, ctypes.POINTER(i32)]
        L.apax_server_release.argtypes = [vp, vp]
        L.apax_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.apax_server_destroy.argtypes = [vp]
        L.apax_server_destroy.restype = None
        L.apax_shard_elements.argtypes = [u64, u32, u64, u64, p64]
        L.apax_encode_shard.argtypes = [vp, i32, u64, pP, u64, u64, vp, u64, vp, u64, vp, vp]
        L.apax_shard_rebase.argtypes = [vp, u64, u64, vp]
        L.apax_merge_shards.argtypes = [ctypes.POINTER(Shard), i32, i32, u64, pP, vp, u64, vp, vp]
        L.apax_quality_workspace_size.argtypes = [i32, u64, p64]
        L.apax_quality_metrics.argtypes = [vp, vp, i32, u64, vp, u64, vp, vp]
        L.apax_quality_db.argtypes = [ctypes.POINTER(Quality), vp]
        L.apax_quality_db.restype = None
        L.apax_status_string.argtypes = [i32]
        L.apax_status_string.restype = ctypes.c_char_p
        L.apax_build_info.argtypes = []
        L.apax_build_info.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        raise ApaxError(st, what)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


_SIDE = {}


def _side_stream(device) -> torch.cuda.Stream:
    """One non-default stream per device for host-to-device copies."""
    key = torch.device(device).index
    if key not in _SIDE:
        _SIDE[key] = torch.cuda.Stream(device=device)
    return _SIDE[key]


def _dtype_code(t: torch.Tensor) -> int:
    try:
        return TORCH_CODE[t.dtype]
    except KeyError:
        raise ApaxError(-3, f"unsupported dtype {t.dtype}") from None


SEARCH_BISECT, SEARCH_PREDICT = 0, 1
# format options (container version 2): BFPE groups of 8, the sum stream
FORMAT_GROUP8, FORMAT_SUM_STREAM = 1, 2


def params(block_size: int = 256, mode: int = FIXED_QUALITY, rate=(4, 1), code: int = 0,
           search: int = SEARCH_BISECT, fmt: int = 0) -> Params:
    return Params(block_size, mode, rate[0], rate[1], code, search, fmt)


def encoded_size(dtype_code: int, n: int, p: Params) -> int:
    out = ctypes.c_uint64()
    _check(lib().apax_encoded_size(dtype_code, n, ctypes.byref(p), ctypes.byref(out)),
           "encoded_size")
    return out.value


def workspace_size(dtype_code: int, n: int, p: Params) -> int:
    out = ctypes.c_uint64()
    _check(lib().apax_workspace_size(dtype_code, n, ctypes.byref(p), ctypes.byref(out)),
           "workspace_size")
    return out.value


def decode_workspace_size() -> int:
    return lib().apax_decode_workspace_size()


def profile_workspace_size(dtype_code: int, n: int, block_size: int, ncand: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().apax_profile_workspace_size(dtype_code, n, block_size, ncand, ctypes.byref(out)),
           "profile_workspace_size")
    return out.value


@dataclass
class Result:
    status: int
    bytes: int


def read_result(res: torch.Tensor) -> Result:
    v = res.view(torch.int64).cpu()
    st = int(v[0].item()) & 0xffffffff
    if st >= 1 << 31:
        st -= 1 << 32
    return Result(st, int(v[1].item()))


def new_result(device) -> torch.Tensor:
    return torch.zeros(RESULT_BYTES, dtype=torch.uint8, device=device)


# ----------------------------------------------------------------- encode
def encode_into(x: torch.Tensor, p: Params, out: torch.Tensor, workspace: torch.Tensor,
                res: torch.Tensor, stream=None, summary: torch.Tensor | None = None):
    """Enqueue an encode of the contiguous device tensor x into out (uint8)."""
    xf = x.reshape(-1)
    code = _dtype_code(xf)
    args = (xf.data_ptr(), code, xf.numel(), ctypes.byref(p))
    tail = (out.data_ptr(), out.numel(), workspace.data_ptr(), workspace.numel(), res.data_ptr(),
            _stream(stream))
    if summary is None:
        _check(lib().apax_encode(*args, *tail), "encode")
    else:
        _check(lib().apax_encode_recommended(*args, summary.data_ptr(), *tail),
               "encode_recommended")


def encode(x: torch.Tensor, block_size: int = 256, mode: int = FIXED_QUALITY, rate=(4, 1),
           code: int = 0, stream=None, search: int = SEARCH_BISECT, fmt: int = 0) -> torch.Tensor:
    """Encode x (device tensor); returns the container as a uint8 tensor.
    fmt: format options (FORMAT_GROUP8 | FORMAT_SUM_STREAM)."""
    assert x.is_cuda and x.is_contiguous()
    p = params(block_size, mode, rate, code, search, fmt)
    dc = _dtype_code(x)
    cap = encoded_size(dc, x.numel(), p)
    out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    ws = torch.empty(workspace_size(dc, x.numel(), p), dtype=torch.uint8, device=x.device)
    res = new_result(x.device)
    encode_into(x, p, out, ws, res, stream)
    r = read_result(res)
    _check(r.status, "encode (device)")
    return out[:r.bytes]


def copy_container_into(out: torch.Tensor, res: torch.Tensor, dst: torch.Tensor, stream=None):
    """Enqueue apax_copy_container: the container in `out` (its size read on
    the device from `res`) into `dst` (a uint8 device tensor or a pinned
    host tensor), with no host round trip."""
    _check(lib().apax_copy_container(out.data_ptr(), res.data_ptr(), dst.data_ptr(), dst.numel(),
                                     _stream(stream)), "copy_container")


def encode_noalloc_into(x: torch.Tensor, p: Params, out: torch.Tensor, res: torch.Tensor,
                        stream=None):
    """Enqueue apax_encode_noalloc: the encode with its scratch in the library's
    fixed device array instead of a caller workspace (for callers that cannot
    allocate).  Overlapping calls share that array and must be serialised."""
    xf = x.reshape(-1)
    _check(lib().apax_encode_noalloc(xf.data_ptr(), _dtype_code(xf), xf.numel(), ctypes.byref(p),
                                     out.data_ptr(), out.numel(), res.data_ptr(),
                                     _stream(stream)), "encode_noalloc")


def encode_status(x: torch.Tensor, p: Params, stream=None) -> Result:
    dc = _dtype_code(x)
    cap = encoded_size(dc, x.numel(), p)
    out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    ws = torch.empty(workspace_size(dc, x.numel(), p), dtype=torch.uint8, device=x.device)
    res = new_result(x.device)
    encode_into(x, p, out, ws, res, stream)
    return read_result(res)


def encode_test_stall(x: torch.Tensor, p: Params, stall_tile: int, spin_cycles: int) -> Result:
    dc = _dtype_code(x)
    cap = encoded_size(dc, x.numel(), p)
    out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    ws = torch.empty(workspace_size(dc, x.numel(), p), dtype=torch.uint8, device=x.device)
    res = new_result(x.device)
    _check(lib().apax_encode_test_stall(x.data_ptr(), dc, x.numel(), ctypes.byref(p),
                                        out.data_ptr(), cap, ws.data_ptr(), ws.numel(),
                                        res.data_ptr(), stall_tile, spin_cycles,
                                        _stream(None)), "encode_test_stall")
    return read_result(res)


# ----------------------------------------------------------------- batches
def encode_jobs(xs, ps, outs, results: torch.Tensor, code_devs=None):
    """ctypes array of apax_encode_job for device tensors xs with params ps,
    containers outs (uint8) and results[i] = bytes [16 i, 16 i + 16) of
    `results`; code_devs[i] (optional) is a device uint32 tensor (or None)."""
    k = len(xs)
    arr = (EncodeJob * k)()
    base = results.data_ptr()
    for i, (x, p, o) in enumerate(zip(xs, ps, outs)):
        xf = x.reshape(-1)
        cd = None if code_devs is None or code_devs[i] is None else code_devs[i].data_ptr()
        arr[i] = EncodeJob(xf.data_ptr(), _dtype_code(xf), 0, xf.numel(), p, cd, o.data_ptr(),
                           o.numel(), base + RESULT_BYTES * i)
    return arr


def read_results(results: torch.Tensor, count: int):
    v = results.view(torch.int64).reshape(-1, 2)[:count].cpu()
    out = []
    for st, nb in v.tolist():
        st &= 0xffffffff
        out.append(Result(st - (1 << 32) if st >= 1 << 31 else st, nb))
    return out


def decode_jobs(containers, ys, block_sizes, results: torch.Tensor):
    """ctypes array of apax_decode_job: containers (uint8 device tensors) into
    ys (device tensors of the original dtype and length)."""
    k = len(containers)
    arr = (DecodeJob * k)()
    base = results.data_ptr()
    for i, (c, y, N) in enumerate(zip(containers, ys, block_sizes)):
        yf = y.reshape(-1)
        arr[i] = DecodeJob(c.data_ptr(), c.numel(), yf.data_ptr(), _dtype_code(yf), N, yf.numel(),
                           base + RESULT_BYTES * i)
    return arr


def profile_jobs(xs, block_sizes, candidates, targets, points, summaries, formats=None):
    """ctypes array of apax_profile_job; candidates[i] is a list of codes (kept
    alive on the returned array), points[i] / summaries[i] device uint8
    tensors (see profile_buffers), formats[i] the format options (default 0)."""
    k = len(xs)
    arr = (ProfileJob * k)()
    arr._keep = []
    for i in range(k):
        xf = xs[i].reshape(-1)
        c = (ctypes.c_uint16 * len(candidates[i]))(*candidates[i])
        arr._keep.append(c)
        fmt = 0 if formats is None else formats[i]
        arr[i] = ProfileJob(xf.data_ptr(), _dtype_code(xf), block_sizes[i], xf.numel(),
                            ctypes.cast(c, ctypes.c_void_p), len(candidates[i]), fmt, targets[i],
                            points[i].data_ptr(), summaries[i].data_ptr())
    return arr


def batch_profile_workspace_size(jobs) -> int:
    out = ctypes.c_uint64()
    _check(lib().apax_batch_profile_workspace_size(jobs, len(jobs), ctypes.byref(out)),
           "batch_profile_workspace_size")
    return out.value


def batch_decode_workspace_size(jobs) -> int:
    out = ctypes.c_uint64()
    _check(lib().apax_batch_decode_workspace_size(jobs, len(jobs), ctypes.byref(out)),
           "batch_decode_workspace_size")
    return out.value


def batch_encode_workspace_size(jobs) -> int:
    out = ctypes.c_uint64()
    _check(lib().apax_batch_encode_workspace_size(jobs, len(jobs), ctypes.byref(out)),
           "batch_encode_workspace_size")
    return out.value


class Batch:
    """A plan running many arrays in one persistent launch (apax_batch_*).
    `jobs` comes from encode_jobs() or decode_jobs(); the tensors behind it
    and `workspace` (a 256-byte aligned uint8 device tensor, see
    batch_*_workspace_size) must outlive the plan."""

    def __init__(self, jobs, workspace: torch.Tensor):
        self.jobs = jobs
        self.workspace = workspace
        h = ctypes.c_void_p()
        if isinstance(jobs[0], ProfileJob):
            _check(lib().apax_batch_profile_create(jobs, len(jobs), workspace.data_ptr(),
                                                   workspace.numel(), ctypes.byref(h)),
                   "batch_profile_create")
        elif isinstance(jobs[0], DecodeJob):
            _check(lib().apax_batch_decode_create(jobs, len(jobs), workspace.data_ptr(),
                                                  workspace.numel(), ctypes.byref(h)),
                   "batch_decode_create")
        else:
            _check(lib().apax_batch_encode_create(jobs, len(jobs), workspace.data_ptr(),
                                                  workspace.numel(), ctypes.byref(h)),
                   "batch_encode_create")
        self.handle = h

    def run(self, stream=None):
        _check(lib().apax_batch_run(self.handle, _stream(stream)), "batch_run")

    def tune(self, reps: int = 3, stream=None):
        _check(lib().apax_batch_tune(self.handle, reps, _stream(stream)), "batch_tune")

    @property
    def config(self):
        c = BatchConfig()
        _check(lib().apax_batch_get_config(self.handle, ctypes.byref(c)), "batch_get_config")
        return (c.threads, c.ctas_per_sm)

    @config.setter
    def config(self, v):
        c = BatchConfig(*v)
        _check(lib().apax_batch_set_config(self.handle, ctypes.byref(c)), "batch_set_config")

    @property
    def tiles(self) -> int:
        return lib().apax_batch_tiles(self.handle)

    def close(self):
        if self.handle:
            lib().apax_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


EncodeBatch = DecodeBatch = ProfileBatch = Batch


def aligned_workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """A uint8 device tensor of nbytes starting on a 256-byte boundary."""
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    return ws[(-ws.data_ptr()) % 256:][:nbytes]


# ----------------------------------------------------------------- serving
class Server:
    """Request server with continuous batching (apax_server_*).  `arena` is a
    256-byte aligned uint8 device tensor: the admission cap and the memory
    outputs the server allocates come from."""

    def __init__(self, arena: torch.Tensor, slots: int = 4, max_batch: int = 256):
        self.arena = arena
        cfg = ServerConfig(arena.data_ptr(), arena.numel(), slots, max_batch)
        h = ctypes.c_void_p()
        _check(lib().apax_server_create(ctypes.byref(cfg), ctypes.byref(h)), "server_create")
        self.handle = h
        self._buf = (Completion * 1024)()

    def submit_encode(self, rid: int, x: torch.Tensor, p: Params, out: torch.Tensor | None = None,
                      t_arrival: float = 0.0):
        xf = x.reshape(-1)
        r = Request(rid, OP_ENCODE, _dtype_code(xf), xf.numel(), p, xf.data_ptr(), 0,
                    out.data_ptr() if out is not None else None,
                    out.numel() if out is not None else 0, t_arrival)
        _check(lib().apax_server_submit(self.handle, ctypes.byref(r)), "server_submit")

    def submit_decode(self, rid: int, container: torch.Tensor, dtype: torch.dtype, n: int,
                      block_size: int, out: torch.Tensor | None = None, t_arrival: float = 0.0):
        p = params(block_size)
        r = Request(rid, OP_DECODE, TORCH_CODE[dtype], n, p, container.data_ptr(),
                    container.numel(), out.data_ptr() if out is not None else None,
                    out.numel() * out.element_size() if out is not None else 0, t_arrival)
        _check(lib().apax_server_submit(self.handle, ctypes.byref(r)), "server_submit")

    def poll(self):
        k = ctypes.c_int()
        _check(lib().apax_server_poll(self.handle, self._buf, len(self._buf), ctypes.byref(k)),
               "server_poll")
        return [Completion.from_buffer_copy(self._buf[i]) for i in range(k.value)]

    def output(self, c: Completion, nbytes: int) -> torch.Tensor:
        """The bytes of a server-allocated output, as a view into the arena."""
        off = c.out - self.arena.data_ptr()
        assert 0 <= off and off + nbytes <= self.arena.numel()
        return self.arena[off:off + nbytes]

    def release(self, out_ptr: int):
        _check(lib().apax_server_release(self.handle, out_ptr), "server_release")

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().apax_server_stats(self.handle, ctypes.byref(st)), "server_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            lib().apax_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- decode
def decode_into(stream_t: torch.Tensor, y: torch.Tensor, workspace: torch.Tensor,
                res: torch.Tensor, stream=None, blocks=None):
    yf = y.reshape(-1)
    code = _dtype_code(yf)
    if blocks is None:
        _check(lib().apax_decode(stream_t.data_ptr(), stream_t.numel(), yf.data_ptr(), code,
                                 yf.numel(), workspace.data_ptr(), workspace.numel(),
                                 res.data_ptr(), _stream(stream)), "decode")
    else:
        b0, b1, n = blocks
        _check(lib().apax_decode_blocks(stream_t.data_ptr(), stream_t.numel(), b0, b1,
                                        yf.data_ptr(), code, n, workspace.data_ptr(),
                                        workspace.numel(), res.data_ptr(), _stream(stream)),
               "decode_blocks")


def decode(stream_t: torch.Tensor, dtype: torch.dtype, n: int, stream=None,
           check: bool = True):
    """Decode a container (uint8 device tensor) into a new tensor of n elements.
    Returns the tensor, or (tensor, Result) when check is False."""
    y = torch.empty(n, dtype=dtype, device=stream_t.device)
    ws = torch.empty(decode_workspace_size(), dtype=torch.uint8, device=stream_t.device)
    res = new_result(stream_t.device)
    try:
        decode_into(stream_t, y, ws, res, stream)
    except ApaxError as e:
        if check:
            raise
        return y, Result(e.status, 0)
    r = read_result(res)
    if check:
        _check(r.status, "decode (device)")
        return y
    return y, r


def decode_blocks(stream_t: torch.Tensor, dtype: torch.dtype, n: int, b0: int, b1: int,
                  block_size: int, stream=None):
    L = min(n, b1 * block_size) - b0 * block_size
    y = torch.empty(max(L, 0), dtype=dtype, device=stream_t.device)
    ws = torch.empty(decode_workspace_size(), dtype=torch.uint8, device=stream_t.device)
    res = new_result(stream_t.device)
    decode_into(stream_t, y, ws, res, stream, blocks=(b0, b1, n))
    r = read_result(res)
    _check(r.status, "decode_blocks (device)")
    return y


# ----------------------------------------------------------------- profile
def profile_into(x: torch.Tensor, block_size: int, candidates, target: float,
                 workspace: torch.Tensor, points: torch.Tensor, summary: torch.Tensor,
                 stream=None, fmt: int = 0):
    """apax_profile (fmt 0) or apax_profile_format (byte counts of the
    containers with those format options)."""
    xf = x.reshape(-1)
    code = _dtype_code(xf)
    if candidates is None:
        cptr, nc = None, 16
    else:
        arr = (ctypes.c_uint16 * len(candidates))(*candidates)
        cptr, nc = ctypes.cast(arr, ctypes.c_void_p), len(candidates)
    tail = (cptr, nc, target, workspace.data_ptr(), workspace.numel(), points.data_ptr(),
            summary.data_ptr(), _stream(stream))
    if fmt:
        _check(lib().apax_profile_format(xf.data_ptr(), code, xf.numel(), block_size, fmt, *tail),
               "profile_format")
    else:
        _check(lib().apax_profile(xf.data_ptr(), code, xf.numel(), block_size, *tail), "profile")


def profile_from_host_into(x_host: torch.Tensor, x_dev: torch.Tensor, block_size: int,
                           candidates, target: float, workspace: torch.Tensor,
                           points: torch.Tensor, summary: torch.Tensor, stream=None,
                           copy_stream=None, chunks: int = 16):
    """apax_profile_from_host: x_host (pinned CPU tensor) is copied into x_dev
    in `chunks` pieces on copy_stream (default: a side stream of this module)
    while the sweep runs on stream."""
    xf, xd = x_host.reshape(-1), x_dev.reshape(-1)
    if copy_stream is None:
        copy_stream = _side_stream(xd.device)
    assert not xf.is_cuda and xd.is_cuda and (xf.numel() == 0 or xf.is_pinned())
    assert xf.dtype == xd.dtype and xf.numel() == xd.numel()
    if candidates is None:
        cptr, nc = None, 16
    else:
        arr = (ctypes.c_uint16 * len(candidates))(*candidates)
        cptr, nc = ctypes.cast(arr, ctypes.c_void_p), len(candidates)
    _check(lib().apax_profile_from_host(xf.data_ptr(), xd.data_ptr(), _dtype_code(xd), xd.numel(),
                                        block_size, cptr, nc, target, chunks,
                                        workspace.data_ptr(), workspace.numel(),
                                        points.data_ptr(), summary.data_ptr(), _stream(stream),
                                        copy_stream.cuda_stream), "profile_from_host")


def profile_buffers(x: torch.Tensor, block_size: int, ncand: int):
    dev = x.device
    ws = torch.empty(profile_workspace_size(_dtype_code(x), x.numel(), block_size, ncand),
                     dtype=torch.uint8, device=dev)
    pts = torch.zeros(POINT_BYTES * ncand, dtype=torch.uint8, device=dev)
    summ = torch.zeros(SUMMARY_BYTES, dtype=torch.uint8, device=dev)
    return ws, pts, summ


def read_points(points: torch.Tensor, ncand: int):
    raw = points.cpu().numpy().tobytes()
    return [Point.from_buffer_copy(raw, i * POINT_BYTES) for i in range(ncand)]


def read_summary(summary: torch.Tensor) -> Summary:
    return Summary.from_buffer_copy(summary.cpu().numpy().tobytes())


def profile(x: torch.Tensor, block_size: int = 256, candidates=DEFAULT_CANDIDATES,
            target: float = 0.99999, stream=None, fmt: int = 0):
    """Returns (points, summary)."""
    nc = len(candidates)
    ws, pts, summ = profile_buffers(x, block_size, nc)
    profile_into(x, block_size, list(candidates), target, ws, pts, summ, stream, fmt)
    return read_points(pts, nc), read_summary(summ)


DERIVED = ("r", "r_centred", "snr_db", "rms_pct", "rms_db", "mean_x", "mean_y", "mean_d",
           "std_x", "std_y", "std_d")


def derived(point: Point, n: int) -> dict:
    out = (ctypes.c_double * 11)()
    lib().apax_derived_metrics(ctypes.byref(point), n, ctypes.cast(out, ctypes.c_void_p))
    return dict(zip(DERIVED, list(out)))


def build_info() -> str:
    return lib().apax_build_info().decode()


# ---------------------------------------------------------------- shards
def shard_elements(n: int, block_size: int, b0: int, b1: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().apax_shard_elements(n, block_size, b0, b1, ctypes.byref(out)), "shard_elements")
    return out.value


def encode_shard(x_halo: torch.Tensor, n: int, p: Params, b0: int, b1: int,
                 stream=None) -> torch.Tensor:
    """Encode blocks [b0, b1) of an array of n elements; x_halo holds those
    blocks' elements preceded by the whole block b0 - 1 when b0 > 0.  Returns
    the shard's container (a container of the sub-array)."""
    assert x_halo.is_cuda and x_halo.is_contiguous()
    dc = _dtype_code(x_halo)
    ns = shard_elements(n, p.block_size, b0, b1)
    cap = encoded_size(dc, ns, p)
    out = torch.empty(cap, dtype=torch.uint8, device=x_halo.device)
    ws = torch.empty(workspace_size(dc, ns, p), dtype=torch.uint8, device=x_halo.device)
    res = new_result(x_halo.device)
    _check(lib().apax_encode_shard(x_halo.data_ptr(), dc, n, ctypes.byref(p), b0, b1,
                                   out.data_ptr(), cap, ws.data_ptr(), ws.numel(), res.data_ptr(),
                                   _stream(stream)), "encode_shard")
    r = read_result(res)
    _check(r.status, "encode_shard (device)")
    return out[:r.bytes]


def shard_rebase(container: torch.Tensor, blocks: int, add_words: int, stream=None):
    _check(lib().apax_shard_rebase(container.data_ptr(), blocks, add_words, _stream(stream)),
           "shard_rebase")


def merge_shards(containers, ranges, dtype_code: int, n: int, p: Params, stream=None) -> torch.Tensor:
    """The whole-array container from shard containers (device tensors) of
    the block ranges `ranges`, in order."""
    k = len(containers)
    arr = (Shard * k)(*[Shard(c.data_ptr(), c.numel(), b0, b1)
                        for c, (b0, b1) in zip(containers, ranges)])
    cap = encoded_size(dtype_code, n, p)
    dev = containers[0].device
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    res = new_result(dev)
    _check(lib().apax_merge_shards(arr, k, dtype_code, n, ctypes.byref(p), out.data_ptr(), cap,
                                   res.data_ptr(), _stream(stream)), "merge_shards")
    r = read_result(res)
    _check(r.status, "merge_shards (device)")
    return out[:r.bytes]


# ---------------------------------------------------------------- quality
def quality_workspace_size(dtype_code: int, n: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().apax_quality_workspace_size(dtype_code, n, ctypes.byref(out)),
           "quality_workspace_size")
    return out.value


def quality_into(x: torch.Tensor, y: torch.Tensor, workspace: torch.Tensor, q: torch.Tensor,
                 stream=None):
    """Enqueue apax_quality_metrics (x, y device tensors of one dtype; q a
    device uint8 tensor of sizeof(Quality) bytes, 8-byte aligned)."""
    xf, yf = x.reshape(-1), y.reshape(-1)
    assert xf.dtype == yf.dtype and xf.numel() == yf.numel()
    _check(lib().apax_quality_metrics(xf.data_ptr(), yf.data_ptr(), _dtype_code(xf), xf.numel(),
                                      workspace.data_ptr(), workspace.numel(), q.data_ptr(),
                                      _stream(stream)), "quality")


def read_quality(q: torch.Tensor) -> Quality:
    b = q.cpu().numpy().tobytes()
    return Quality.from_buffer_copy(b[:ctypes.sizeof(Quality)])


def quality_db(qr: Quality) -> dict:
    import numpy as _np
    out = _np.zeros(len(QUALITY_DB), dtype=_np.float64)
    lib().apax_quality_db(ctypes.byref(qr), out.ctypes.data)
    return dict(zip(QUALITY_DB, out.tolist()))


def quality(x: torch.Tensor, y: torch.Tensor, stream=None):
    """(Quality record, its levels in dB) for x against y."""
    ws = aligned_workspace(quality_workspace_size(_dtype_code(x.reshape(-1)), x.numel()),
                           x.device)
    q = torch.zeros(ctypes.sizeof(Quality), dtype=torch.uint8, device=x.device)
    quality_into(x, y, ws, q, stream)
    qr = read_quality(q)
    return qr, quality_db(qr)
