"""Python binding of libsgs.so (ctypes).  Argument marshalling only: every step of the decode
path runs in the library's CUDA kernels; there is no Python or CPU fallback.  Names follow the
C ABI in include/sgs.h.  Device buffers are passed as torch CUDA tensors or raw pointers;
streams as torch.cuda.Stream, a raw cudaStream_t int, or None (the current torch stream)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, E_INVALID, E_CORRUPT, E_NOMEM, E_CUDA, E_TIMEOUT, E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
MODE_FIXED, MODE_STATIC, MODE_LEARNED, MODE_LEARNED_PE = 0, 1, 2, 3
GEO_RAW, GEO_RANS, GEO_LEARNED = 0, 1, 2
NCHAN = 56
MAX_DEPTH = 21
MODEL_BYTES = 36384
MODEL_PE_BYTES = 23984
WEIGHTS_FLOATS = 56 * 16 + 64 * 20 + 64 + 64 * 64 + 64 + 256 * 64 + 256
WEIGHTS_PE_FLOATS = 56 * 16 + 32 * 75 + 32 + 64 * 52 + 64 + 64 * 64 + 64 + 2 * 64 + 2

u32, u64, i32, P = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p


class SceneInfo(ctypes.Structure):
    _fields_ = [("mode", u32), ("geo_mode", u32), ("n_in", u32), ("n_rows", u32), ("depth", u32),
                ("n_leaves", u32), ("n_dup", u32), ("lanes", u32), ("geo_lanes", u32),
                ("n_level", u32 * (MAX_DEPTH + 1)), ("n_geo", u64), ("n_geo_coded", u64),
                ("off", u64 * 11), ("total_len", u64), ("scratch_bytes", u64),
                ("n_tables", u32), ("table_off", u32 * (NCHAN + MAX_DEPTH))]


class SceneOut(ctypes.Structure):
    _fields_ = [("attr", P), ("pos", P), ("coord", P), ("out_index", P)]


class EncodeParams(ctypes.Structure):
    _fields_ = [("mode", u32), ("geo_mode", u32), ("depth", u32), ("lanes", u32), ("geo_lanes", u32),
                ("bits", u32 * NCHAN), ("model", P), ("geo_model", P)]


class TrainParams(ctypes.Structure):
    _fields_ = [("steps", u32), ("batch", u32), ("seed", u32), ("lr", ctypes.c_float)]


TUNE_MAX_CAND = 16


class TuneRequest(ctypes.Structure):
    _fields_ = [("pos", P), ("attr", P), ("n", u32), ("mode", u32), ("depth", u32), ("geo_mode", u32),
                ("model", P), ("n_cand", u32), ("rows_per_lane", u32 * TUNE_MAX_CAND), ("max_ms", ctypes.c_float),
                ("reps", u32), ("n_shape", u32), ("warps_per_cta", u32 * TUNE_MAX_CAND)]


class TuneResult(ctypes.Structure):
    _fields_ = [("best", u32), ("lanes", u32 * TUNE_MAX_CAND), ("bytes", u64 * TUNE_MAX_CAND),
                ("ms", ctypes.c_float * TUNE_MAX_CAND),
                ("warps", u32 * TUNE_MAX_CAND), ("best_warps", u32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("bits_dev", P), ("info", SceneInfo), ("out", SceneOut)]


class Camera(ctypes.Structure):
    _fields_ = [("rot", ctypes.c_float * 9), ("origin", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", u32),
                ("height", u32)]


class SgsError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s: %s (%d)" % (what, lib().sgs_strerror(code).decode(), code))
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libsgs.so (building it first if the sources are newer).  Raises if it cannot."""
    global _lib
    if _lib is None:
        path = os.environ.get("SGS_LIBRARY")  # an alternative build of the same library
        if not path:
            path = _build.LIB
            if not os.path.exists(path) or _build.needs_build():
                path = _build.build()
        L = ctypes.CDLL(path)
        L.sgs_strerror.restype = ctypes.c_char_p
        L.sgs_strerror.argtypes = [i32]
        L.sgs_create.argtypes = [ctypes.POINTER(P), i32, ctypes.c_size_t]
        L.sgs_reserve.argtypes = [P, ctypes.c_size_t]
        L.sgs_destroy.argtypes = [P]
        L.sgs_destroy.restype = None
        L.sgs_sync.argtypes = [P, P]
        L.scene_query.argtypes = [P, ctypes.c_size_t, ctypes.POINTER(SceneInfo)]
        L.scene_decode.argtypes = [P, P, ctypes.POINTER(SceneInfo), ctypes.POINTER(SceneOut), P]
        L.scene_decode_batch.argtypes = [P, ctypes.POINTER(BatchItem), i32, P]
        L.scene_batch_bytes.argtypes = [ctypes.POINTER(BatchItem), i32, ctypes.POINTER(ctypes.c_size_t)]
        L.scene_batch_plan.argtypes = [P, ctypes.POINTER(BatchItem), i32, ctypes.POINTER(P)]
        L.scene_batch_run.argtypes = [P, P, P]
        L.scene_batch_status.argtypes = [P, ctypes.POINTER(i32), i32]
        L.scene_batch_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), i32]
        L.scene_batch_free.argtypes = [P]
        L.scene_batch_free.restype = None
        L.scene_encode.argtypes = [P, P, P, u32, ctypes.POINTER(EncodeParams), P, ctypes.c_size_t,
                                   ctypes.POINTER(ctypes.c_size_t)]
        L.scene_tokens.argtypes = [P, P, u32, u32, P, ctypes.c_size_t, ctypes.POINTER(u32)]
        L.scene_rows.argtypes = [P, P, u32, u32, P, P, u32, ctypes.POINTER(u32)]
        L.scene_geo_samples.argtypes = [P, P, u32, u32, P, P, P, u64, ctypes.POINTER(u64)]
        L.sgs_render.argtypes = [P, P, P, u32, ctypes.POINTER(Camera), P, P]
        L.sgs_train_pe.argtypes = [P, P, P, u32, u32, u32, ctypes.POINTER(TrainParams), u32, P, P, P]
        L.sgs_train_pe_grad.argtypes = [P, P, P, u32, u32, u32, P, u32, P, P, ctypes.POINTER(ctypes.c_float)]
        L.sgs_freeze_pe.argtypes = [P, P, P, u32, u32, u32, u32, P]
        L.sgs_train.argtypes = [P, P, u32, u32, ctypes.POINTER(TrainParams), u32, P, P, P]
        L.sgs_train_grad.argtypes = [P, P, u32, u32, P, u32, P, P, ctypes.POINTER(ctypes.c_float)]
        L.sgs_freeze.argtypes = [P, P, u32, u32, u32, P]
        L.sgs_freeze_samples.argtypes = [P, P, P, u64, u32, P]
        L.sgs_profile.argtypes = [P, i32]
        L.sgs_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_float), i32]
        L.sgs_launch_count.argtypes = [P]
        L.sgs_launch_count.restype = u64
        L.sgs_set_wait_limit.argtypes = [P, u32]
        L.sgs_set_launch_shape.argtypes = [P, u32, u32]
        L.scene_decode_noalloc.argtypes = [P, ctypes.POINTER(SceneInfo), ctypes.POINTER(SceneOut), P]
        L.sgs_autotune.argtypes = [P, ctypes.POINTER(TuneRequest), ctypes.POINTER(TuneResult)]
        _lib = L
    return _lib


def _check(code: int, what: str) -> int:
    if code != OK:
        raise SgsError(code, what)
    return code


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    raise TypeError("expected a tensor, array or pointer")


def _stream(s) -> int:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ----------------------------------------------------------------------------- context

class Context:
    """Owns an sgs_ctx (device scratch, status word) on one CUDA device."""

    def __init__(self, device: int = 0, scratch_bytes: int = 0):
        h = P()
        _check(lib().sgs_create(ctypes.byref(h), device, scratch_bytes), "sgs_create")
        self.handle = h
        self.device = device
        self.scratch_bytes = scratch_bytes

    def reserve(self, nbytes: int) -> None:
        if nbytes > self.scratch_bytes:
            _check(lib().sgs_reserve(self.handle, nbytes), "sgs_reserve")
            self.scratch_bytes = nbytes

    def sync(self, stream=None) -> int:
        """Waits for the stream; returns (and clears) the worst device status since last sync."""
        return lib().sgs_sync(self.handle, _stream(stream))

    def profile(self, enable: bool = True) -> None:
        _check(lib().sgs_profile(self.handle, int(enable)), "sgs_profile")

    def profile_read(self) -> list:
        """[geometry tokens, octree + positions, attributes (own stream), whole decode] ms of
        the last profiled decode."""
        ms = (ctypes.c_float * 4)()
        _check(lib().sgs_profile_read(self.handle, ms, 4), "sgs_profile_read")
        return [float(v) for v in ms]

    def launch_count(self) -> int:
        return int(lib().sgs_launch_count(self.handle))

    def set_launch_shape(self, mode: int, warps_per_cta: int) -> None:
        """Warps per CTA of the attribute decoder for this context's decodes of `mode`
        (fixed-length 1..8, static 1..32; 0 = the built-in shape)."""
        _check(lib().sgs_set_launch_shape(self.handle, mode, warps_per_cta), "sgs_set_launch_shape")

    def set_wait_limit(self, polls: int) -> None:
        """Poll budget of the learned decoders' bounded device waits (0 = the default)."""
        _check(lib().sgs_set_wait_limit(self.handle, polls), "sgs_set_wait_limit")

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().sgs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sgs_create(device: int = 0, scratch_bytes: int = 0) -> Context:
    return Context(device, scratch_bytes)


def sgs_sync(ctx: Context, stream=None) -> int:
    return ctx.sync(stream)


# ----------------------------------------------------------------------------- decode

def scene_query(bits: bytes) -> SceneInfo:
    info = SceneInfo()
    buf = np.frombuffer(bits, np.uint8)
    _check(lib().scene_query(buf.ctypes.data, len(bits), ctypes.byref(info)), "scene_query")
    return info


def _out(attr, pos, coord=None, out_index=None) -> SceneOut:
    return SceneOut(_ptr(attr), _ptr(pos), _ptr(coord), _ptr(out_index))


def scene_decode(ctx: Context, bits_dev, info: SceneInfo, attr, pos, coord=None, out_index=None,
                 stream=None) -> None:
    """Enqueues the decode of one scene (bits_dev: device uint8 tensor of the bitstream)."""
    out = _out(attr, pos, coord, out_index)
    _check(lib().scene_decode(ctx.handle, _ptr(bits_dev), ctypes.byref(info), ctypes.byref(out),
                              _stream(stream)), "scene_decode")


def _header_constant(name: str) -> int:
    """An integer #define of the library's C header (include/sgs.h), so that the binding
    never restates a size the library fixes."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sgs.h")
    m = re.search(r"^#define\s+%s\s+(.+?)\s*(/\*.*)?$" % name, open(hdr).read(), re.M)
    if not m:
        raise RuntimeError("%s is not defined in %s" % (name, hdr))
    expr = re.sub(r"(?<=\d)[uU]?[lL]{0,2}\b", "", m.group(1))
    if not re.fullmatch(r"[\d\s()<+*-]+", expr):
        raise RuntimeError("cannot evaluate %s = %s" % (name, m.group(1)))
    return int(eval(expr, {"__builtins__": {}}))


NOALLOC_SCRATCH_BYTES = _header_constant("SGS_NOALLOC_SCRATCH_BYTES")


def scene_decode_noalloc(bits_dev, info: SceneInfo, attr, pos, coord=None, out_index=None,
                         stream=None) -> int:
    """Decodes one scene with the library's fixed scratch array (no allocation, no context);
    synchronous; returns the decode status (raises on argument or size errors)."""
    out = _out(attr, pos, coord, out_index)
    code = lib().scene_decode_noalloc(_ptr(bits_dev), ctypes.byref(info), ctypes.byref(out),
                                      _stream(stream))
    if code in (E_INVALID, E_NOMEM, E_CUDA, E_UNSUPPORTED):
        raise SgsError(code, "scene_decode_noalloc")
    return code


def _batch_items(items: list):
    """items: (bits_dev, info, attr, pos[, coord[, out_index]]) tuples -> a BatchItem array."""
    arr = (BatchItem * max(len(items), 1))()
    for i, it in enumerate(items):
        bits_dev, info, attr, pos = it[:4]
        coord = it[4] if len(it) > 4 else None
        oidx = it[5] if len(it) > 5 else None
        arr[i].bits_dev = _ptr(bits_dev)
        arr[i].info = info
        arr[i].out = _out(attr, pos, coord, oidx)
    return arr


def scene_batch_bytes(items: list) -> int:
    """Device bytes of a batch plan (every scene's scratch plus the work lists)."""
    n = ctypes.c_size_t(0)
    _check(lib().scene_batch_bytes(_batch_items(items), len(items), ctypes.byref(n)), "scene_batch_bytes")
    return n.value


def scene_decode_batch(ctx: Context, items: list, stream=None) -> None:
    """One-shot batched decode in the context's scratch (needs scene_batch_bytes(items))."""
    _check(lib().scene_decode_batch(ctx.handle, _batch_items(items), len(items), _stream(stream)),
           "scene_decode_batch")


class BatchPlan:
    """A batched decode plan: binds the items' buffers; run() enqueues one decode of all of
    them (no allocation, no host wait: capturable in a CUDA graph)."""

    def __init__(self, ctx: Context, items: list):
        h = P()
        _check(lib().scene_batch_plan(ctx.handle, _batch_items(items), len(items), ctypes.byref(h)),
               "scene_batch_plan")
        self.handle = h
        self.ctx = ctx
        self.n = len(items)
        self.items = items  # keep the bound buffers alive

    def run(self, stream=None) -> None:
        _check(lib().scene_batch_run(self.ctx.handle, self.handle, _stream(stream)), "scene_batch_run")

    def status(self) -> list[int]:
        arr = (i32 * max(self.n, 1))()
        _check(lib().scene_batch_status(self.handle, arr, self.n), "scene_batch_status")
        return list(arr[:self.n])

    def times_ms(self) -> list[float]:
        """Per-scene completion times (ms from the start of the last finished run; -1 for a
        scene without work)."""
        arr = (ctypes.c_double * max(self.n, 1))()
        _check(lib().scene_batch_times(self.handle, arr, self.n), "scene_batch_times")
        return list(arr[:self.n])

    def close(self) -> None:
        if self.handle:
            lib().scene_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- encode

def scene_encode(pos: np.ndarray, attr: np.ndarray, *, mode: int, depth: int, lanes: int = 32,
                 geo_mode: int = GEO_RANS, geo_lanes: int = 0, bits=8, model: bytes | None = None,
                 ctx: Context | None = None, geo_model: bytes | None = None) -> bytes:
    pos = np.ascontiguousarray(pos, np.float32)
    attr = np.ascontiguousarray(attr, np.float32)
    n = pos.shape[1]
    assert pos.shape == (3, n) and attr.shape == (NCHAN, n)
    prm = EncodeParams()
    prm.mode, prm.geo_mode, prm.depth, prm.lanes, prm.geo_lanes = mode, geo_mode, depth, lanes, geo_lanes
    b = np.broadcast_to(np.asarray(bits, np.uint32), (NCHAN,))
    for c in range(NCHAN):
        prm.bits[c] = int(b[c])
    mbuf = None
    if model is not None:
        mbuf = np.frombuffer(bytes(model), np.uint8).copy()
        assert mbuf.size == (MODEL_PE_BYTES if mode == MODE_LEARNED_PE else MODEL_BYTES)
        prm.model = mbuf.ctypes.data
    gbuf = None
    if geo_model is not None:
        gbuf = np.frombuffer(bytes(geo_model), np.uint8).copy()
        assert gbuf.size == MODEL_BYTES
        prm.geo_model = gbuf.ctypes.data
    need = ctypes.c_size_t(0)
    h = ctx.handle if ctx is not None else None
    # one pass in the common case: room for 2 bytes per token plus tables and headers
    cap = (1 << 20) + n * (2 * NCHAN + 16) + 64 * (lanes + geo_lanes)
    out = np.empty(cap, np.uint8)
    code = lib().scene_encode(h, pos.ctypes.data, attr.ctypes.data, n, ctypes.byref(prm), out.ctypes.data,
                              out.size, ctypes.byref(need))
    if code == E_INVALID and need.value > cap:
        out = np.empty(need.value, np.uint8)
        code = lib().scene_encode(h, pos.ctypes.data, attr.ctypes.data, n, ctypes.byref(prm),
                                  out.ctypes.data, out.size, ctypes.byref(need))
    _check(code, "scene_encode")
    return out[: need.value].tobytes()


def scene_tokens(pos: np.ndarray, attr: np.ndarray, depth: int) -> np.ndarray:
    """uint8 [n_rows][56] quantized tokens, rows in Morton order (8-bit channels)."""
    pos = np.ascontiguousarray(pos, np.float32)
    attr = np.ascontiguousarray(attr, np.float32)
    n = pos.shape[1]
    tok = np.zeros((n, NCHAN), np.uint8)
    nr = u32(0)
    _check(lib().scene_tokens(pos.ctypes.data, attr.ctypes.data, n, depth, tok.ctypes.data, tok.size,
                              ctypes.byref(nr)), "scene_tokens")
    return tok[: nr.value].copy()


def scene_geo_samples(pos: np.ndarray, attr: np.ndarray, depth: int):
    """The learned geometry coder's training samples: (u int32 [n, 4], chan uint32 [n],
    sym uint8 [n]) over the nodes of every coded octree level."""
    pos = np.ascontiguousarray(pos, np.float32)
    attr = np.ascontiguousarray(attr, np.float32)
    n = pos.shape[1]
    need = u64(0)
    code = lib().scene_geo_samples(pos.ctypes.data, attr.ctypes.data, n, depth, None, None, None, 0,
                                   ctypes.byref(need))
    if code != OK and not (code == E_INVALID and need.value > 0):
        _check(code, "scene_geo_samples")
    k = need.value
    uu = np.zeros((max(k, 1), 4), np.int32)
    cc = np.zeros(max(k, 1), np.uint32)
    ss = np.zeros(max(k, 1), np.uint8)
    _check(lib().scene_geo_samples(pos.ctypes.data, attr.ctypes.data, n, depth, uu.ctypes.data, cc.ctypes.data,
                                   ss.ctypes.data, k, ctypes.byref(need)), "scene_geo_samples")
    return uu[:k], cc[:k], ss[:k]


def scene_rows(pos: np.ndarray, attr: np.ndarray, depth: int):
    """(tokens uint8 [n_rows, 56], voxel coordinates uint32 [3, n_rows]) as the encoder sees
    the rows."""
    pos = np.ascontiguousarray(pos, np.float32)
    attr = np.ascontiguousarray(attr, np.float32)
    n = pos.shape[1]
    tok = np.zeros((max(n, 1), NCHAN), np.uint8)
    crd = np.zeros(3 * max(n, 1), np.uint32)
    nr = u32(0)
    _check(lib().scene_rows(pos.ctypes.data, attr.ctypes.data, n, depth, tok.ctypes.data, crd.ctypes.data,
                            max(n, 1), ctypes.byref(nr)), "scene_rows")
    r = nr.value
    return tok[:r].copy(), crd[:3 * r].reshape(3, r).copy()


def camera(rot, origin, fx: float, fy: float, cx: float, cy: float, width: int, height: int) -> Camera:
    c = Camera()
    for i, v in enumerate(np.asarray(rot, np.float32).ravel()):
        c.rot[i] = float(v)
    for i, v in enumerate(np.asarray(origin, np.float32).ravel()):
        c.origin[i] = float(v)
    c.fx, c.fy, c.cx, c.cy, c.width, c.height = fx, fy, cx, cy, width, height
    return c


def look_at(origin, target, up, width: int, height: int, fov_y_deg: float) -> Camera:
    """A pinhole camera at `origin` looking at `target`, vertical field of view fov_y_deg
    (camera axes: x right, y down, z forward)."""
    o = np.asarray(origin, np.float64)
    z = np.asarray(target, np.float64) - o
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    f = 0.5 * height / np.tan(np.radians(fov_y_deg) / 2)
    return camera(np.stack([x, y, z]), o, f, f, width / 2.0, height / 2.0, width, height)


def render(ctx: Context, attr_dev, pos_dev, n: int, cam: Camera, image_dev, stream=None) -> None:
    """Splats n decoded Gaussians into image_dev (device float [3, height, width])."""
    _check(lib().sgs_render(ctx.handle, _ptr(attr_dev), _ptr(pos_dev), n, ctypes.byref(cam), _ptr(image_dev),
                            _stream(stream)), "sgs_render")


# ----------------------------------------------------------------------------- learned part

def sgs_train(ctx: Context, tokens_dev, n_rows: int, lanes: int, weights_dev, adam_dev, *, steps: int,
              batch: int = 65536, seed: int = 0, lr: float = 1e-3, step0: int = 0, loss_dev=None) -> None:
    prm = TrainParams(steps, batch, seed, lr)
    _check(lib().sgs_train(ctx.handle, _ptr(tokens_dev), n_rows, lanes, ctypes.byref(prm), step0,
                           _ptr(weights_dev), _ptr(adam_dev), _ptr(loss_dev)), "sgs_train")


def sgs_train_grad(ctx: Context, tokens_dev, n_rows: int, lanes: int, pos_dev, weights_dev, grad_dev) -> float:
    loss = ctypes.c_float(0)
    n = int(pos_dev.numel()) if hasattr(pos_dev, "numel") else len(pos_dev)
    _check(lib().sgs_train_grad(ctx.handle, _ptr(tokens_dev), n_rows, lanes, _ptr(pos_dev), n,
                                _ptr(weights_dev), _ptr(grad_dev), ctypes.byref(loss)), "sgs_train_grad")
    return float(loss.value)


def sgs_freeze(weights: np.ndarray, tokens: np.ndarray, lanes: int, seed: int) -> bytes:
    w = np.ascontiguousarray(weights, np.float32)
    assert w.size == WEIGHTS_FLOATS
    t = np.ascontiguousarray(tokens, np.uint8)
    out = np.zeros(MODEL_BYTES, np.uint8)
    _check(lib().sgs_freeze(w.ctypes.data, t.ctypes.data, t.shape[0], lanes, seed, out.ctypes.data),
           "sgs_freeze")
    return out.tobytes()


def sgs_freeze_samples(weights: np.ndarray, u: np.ndarray, chan: np.ndarray, seed: int) -> bytes:
    """Frozen integer model (SGS_MODEL_BYTES) from fp32 weights and an explicit sample set of
    contexts u [n, 4] (int, in [-128, 127]) and channels chan [n]."""
    w = np.ascontiguousarray(weights, np.float32)
    assert w.size == WEIGHTS_FLOATS
    uu = np.ascontiguousarray(u, np.int32)
    cc = np.ascontiguousarray(chan, np.uint32)
    assert uu.ndim == 2 and uu.shape[1] == 4 and cc.shape == (uu.shape[0],)
    out = np.zeros(MODEL_BYTES, np.uint8)
    _check(lib().sgs_freeze_samples(w.ctypes.data, uu.ctypes.data, cc.ctypes.data, cc.size, seed, out.ctypes.data),
           "sgs_freeze_samples")
    return out.tobytes()


def sgs_train_pe(ctx: Context, tokens_dev, coord_dev, depth: int, n_rows: int, lanes: int, weights_dev, adam_dev,
                 *, steps: int, batch: int = 65536, seed: int = 0, lr: float = 1e-3, step0: int = 0,
                 loss_dev=None) -> None:
    prm = TrainParams(steps, batch, seed, lr)
    _check(lib().sgs_train_pe(ctx.handle, _ptr(tokens_dev), _ptr(coord_dev), depth, n_rows, lanes,
                              ctypes.byref(prm), step0, _ptr(weights_dev), _ptr(adam_dev), _ptr(loss_dev)),
           "sgs_train_pe")


def sgs_train_pe_grad(ctx: Context, tokens_dev, coord_dev, depth: int, n_rows: int, lanes: int, pos_dev,
                      weights_dev, grad_dev) -> float:
    loss = ctypes.c_float(0)
    n = int(pos_dev.numel())
    _check(lib().sgs_train_pe_grad(ctx.handle, _ptr(tokens_dev), _ptr(coord_dev), depth, n_rows, lanes,
                                   _ptr(pos_dev), n, _ptr(weights_dev), _ptr(grad_dev), ctypes.byref(loss)),
           "sgs_train_pe_grad")
    return float(loss.value)


def sgs_freeze_pe(weights: np.ndarray, tokens: np.ndarray, coord: np.ndarray, depth: int, lanes: int,
                  seed: int) -> bytes:
    w = np.ascontiguousarray(weights, np.float32)
    assert w.size == WEIGHTS_PE_FLOATS
    t = np.ascontiguousarray(tokens, np.uint8)
    c = np.ascontiguousarray(coord, np.uint32)
    assert c.shape == (3, t.shape[0])
    out = np.zeros(MODEL_PE_BYTES, np.uint8)
    _check(lib().sgs_freeze_pe(w.ctypes.data, t.ctypes.data, c.ctypes.data, depth, t.shape[0], lanes, seed,
                               out.ctypes.data), "sgs_freeze_pe")
    return out.tobytes()


WEIGHT_PE_SHAPES = [("emb", (56, 16)), ("wp", (32, 75)), ("bp", (32,)), ("w1", (64, 52)), ("b1", (64,)),
                    ("w2", (64, 64)), ("b2", (64,)), ("w3", (2, 64)), ("b3", (2,))]


def pack_weights_pe(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], np.float32).reshape(-1) for k, _ in WEIGHT_PE_SHAPES])


def unpack_weights_pe(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for k, shp in WEIGHT_PE_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], np.float32).reshape(shp)
        o += n
    return out


WEIGHT_SHAPES = [("emb", (56, 16)), ("w1", (64, 20)), ("b1", (64,)), ("w2", (64, 64)), ("b2", (64,)),
                 ("w3", (256, 64)), ("b3", (256,))]


def pack_weights(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], np.float32).reshape(-1) for k, _ in WEIGHT_SHAPES])


def unpack_weights(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for k, shp in WEIGHT_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], np.float32).reshape(shp)
        o += n
    return out


# ----------------------------------------------------------------------------- autotuning

def autotune(ctx: Context, pos: np.ndarray, attr: np.ndarray, *, mode: int, depth: int, rows_per_lane,
             max_ms: float = 0.0, reps: int = 5, geo_mode: int = GEO_RANS, model: bytes | None = None,
             warps_per_cta=()) -> dict:
    """Encodes the scene at every candidate W (rows per lane), times each decode on the
    context's device (at every candidate launch shape, keeping the fastest) and returns
    {"best": index, "lanes": [...], "bytes": [...], "ms": [...], "warps": [...], "best_warps": w}."""
    pos = np.ascontiguousarray(pos, np.float32)
    attr = np.ascontiguousarray(attr, np.float32)
    cands = list(rows_per_lane)
    assert 1 <= len(cands) <= TUNE_MAX_CAND
    rq = TuneRequest()
    rq.pos, rq.attr, rq.n = pos.ctypes.data, attr.ctypes.data, pos.shape[1]
    rq.mode, rq.depth, rq.geo_mode = mode, depth, geo_mode
    mbuf = None
    if model is not None:
        mbuf = np.frombuffer(bytes(model), np.uint8).copy()
        rq.model = mbuf.ctypes.data
    rq.n_cand = len(cands)
    for i, w in enumerate(cands):
        rq.rows_per_lane[i] = int(w)
    rq.max_ms, rq.reps = max_ms, reps
    shapes = list(warps_per_cta)
    assert len(shapes) <= TUNE_MAX_CAND
    rq.n_shape = len(shapes)
    for i, w in enumerate(shapes):
        rq.warps_per_cta[i] = int(w)
    res = TuneResult()
    _check(lib().sgs_autotune(ctx.handle, ctypes.byref(rq), ctypes.byref(res)), "sgs_autotune")
    k = len(cands)
    return {"best": int(res.best), "rows_per_lane": cands, "lanes": list(res.lanes[:k]),
            "bytes": [int(b) for b in res.bytes[:k]], "ms": list(res.ms[:k]), "warps": list(res.warps[:k]),
            "best_warps": int(res.best_warps)}
