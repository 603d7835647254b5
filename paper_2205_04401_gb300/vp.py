"""Python binding of libvp (include/vp.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module only turns
torch tensors into pointers and status codes into exceptions.  There is no
CPU fallback: if libvp cannot be built or loaded, or no sm_103 GPU is
present, the calls raise.

    ctx  = Context(0)
    mesh = mesh_upload(ctx, vxy, tri, rule=19)             # host numpy arrays
    nf   = nearfield_build(ctx, mesh, node_targets=True, txy=extra_dev)
    u    = potential_eval(ctx, nf, f_dev, precision=VP_MIXED)   # f_dev: [d][N] cuda float64
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

VP_OK = 0
VP_RULE_16_D8 = 16
VP_RULE_19_D9 = 19
VP_RULE_CONICAL_MIN = 8
VP_RULE_CONICAL_MAX = 50


VP_RULE_SYM_DEGREES = (12, 20, 25, 30, 40, 50)


def VP_RULE_CONICAL(n: int) -> int:
    """Rule code of the conical-product Gauss far rule of total degree n (vp.h)."""
    return 1000 + int(n)


def VP_RULE_SYM(n: int) -> int:
    """Rule code of the tabulated S3-symmetric far rule of degree n (vp.h)."""
    return 2000 + int(n)


VP_FP64 = 0
VP_MIXED = 1
VP_MIXED_TC = 2
VP_MIXED_FMM = 3

_lib = None


class VPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} ({code})")
        self.code = code


class NfParams(C.Structure):
    _fields_ = [("eps", C.c_double), ("c_far", C.c_double), ("c_near", C.c_double),
                ("depth_cap", C.c_int32), ("flags", C.c_int32)]


class NfStats(C.Structure):
    _fields_ = [("n_targets", C.c_int64), ("n_nodes", C.c_int64), ("n_pairs", C.c_int64), ("n_self", C.c_int64),
                ("n_near", C.c_int64), ("near_leaves", C.c_int64), ("self_panels", C.c_int64),
                ("depth_capped", C.c_int64), ("outside", C.c_int64), ("bytes_device", C.c_int64),
                ("build_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("queued", C.c_int64), ("cold_builds", C.c_int64),
                ("evals", C.c_int64), ("peak_bytes", C.c_int64), ("max_concurrent", C.c_int32),
                ("reserved", C.c_int32), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("p50_wait_ms", C.c_double), ("evals_per_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class EvalItem(C.Structure):
    _fields_ = [("nf", C.c_void_p), ("f_dev", C.c_void_p), ("d", C.c_int32), ("u_dev", C.c_void_p)]


SIGNATURES = {
    "vp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "vp_destroy": (None, [C.c_void_p]),
    "vp_ctx_memory": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "vp_set_far_sym_cap": (C.c_int, [C.c_void_p, C.c_int64]),
    "vp_status_str": (C.c_char_p, [C.c_int]),
    "vp_last_error": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int32]),
    "vp_mesh_upload": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    "vp_mesh_upload_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32,
                                     C.c_void_p, C.POINTER(C.c_void_p)]),
    "vp_mesh_upload_curved": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p,
                                        C.POINTER(C.c_void_p)]),
    "vp_interp_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                   C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "vp_interp_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "vp_interp_nodes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vp_interp_coeffs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "vp_interp_eval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "vp_interp_release": (None, [C.c_void_p]),
    "vp_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "vp_profile_reset": (C.c_int, [C.c_void_p]),
    "vp_profile_read": (C.c_int, [C.c_void_p, C.c_char_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "vp_mesh_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "vp_mesh_nodes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vp_mesh_release": (None, [C.c_void_p]),
    "vp_nearfield_build": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.POINTER(NfParams),
                                     C.c_void_p, C.POINTER(C.c_void_p)]),
    "vp_nf_stats": (C.c_int, [C.c_void_p, C.POINTER(NfStats)]),
    "vp_nearfield_build_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int64,
                                          C.POINTER(NfParams), C.c_void_p, C.POINTER(C.c_void_p)]),
    "vp_nf_params_default": (C.c_int, [C.POINTER(NfParams)]),
    "vp_nf_lists": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vp_nf_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vp_nf_release": (None, [C.c_void_p]),
    "vp_nf_prepare_tc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "vp_nf_tc_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64)]),
    "vp_device_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vp_nf_fmm_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "vp_potential_eval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]),
    "vp_potential_eval_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                            C.c_void_p]),
    "vp_potential_eval_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                         C.c_void_p]),
    "vp_potential_eval_batch": (C.c_int, [C.c_void_p, C.POINTER(EvalItem), C.c_int32, C.c_int32, C.c_void_p]),
    "vp_batch_create": (C.c_int, [C.c_void_p, C.POINTER(EvalItem), C.c_int32, C.c_int32, C.c_void_p,
                                  C.POINTER(C.c_void_p)]),
    "vp_batch_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vp_batch_release": (None, [C.c_void_p]),
    "vp_set_batch_tile": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "vp_batch_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vp_server_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_void_p)]),
    "vp_server_register": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "vp_server_register_cold": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                          C.c_int32]),
    "vp_server_mesh_size": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "vp_server_submit": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int64)]),
    "vp_server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "vp_server_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "vp_server_destroy": (None, [C.c_void_p]),
    "vp_rule_table": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int32,
                                C.POINTER(C.c_int32)]),
    "vp_far_rule": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                              C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libvp (building it first if its sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libvp not found at {_build.LIB}; run paper_2205_04401_gb300/build.py")
    lib = C.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, ctx=None, what=""):
    if rc == VP_OK:
        return
    lib = load()
    msg = lib.vp_status_str(rc).decode()
    if ctx is not None and ctx.handle:
        buf = C.create_string_buffer(512)
        lib.vp_last_error(ctx.handle, buf, 512)
        msg += ": " + buf.value.decode()
    raise VPError(rc, f"{what}: {msg}")


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, dtype_name):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"expected a CUDA tensor ({dtype_name})")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected torch.{dtype_name}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


class Context:
    """A libvp context on one CUDA device (vp_create / vp_destroy)."""

    def __init__(self, device: int = 0):
        lib = load()
        h = C.c_void_p()
        rc = lib.vp_create(C.byref(h), int(device))
        if rc != VP_OK:
            raise VPError(rc, f"vp_create(device={device}): {lib.vp_status_str(rc).decode()}")
        self.handle = h
        self.device = device

    def memory(self) -> dict:
        """vp_ctx_memory: device bytes of the context's evaluation workspace and staging buffer."""
        ws, st = C.c_int64(), C.c_int64()
        _check(load().vp_ctx_memory(self.handle, C.byref(ws), C.byref(st)), self, "vp_ctx_memory")
        return {"workspace_bytes": ws.value, "staging_bytes": st.value}

    def set_batch_tile(self, width: int, targets_per_thread: int):
        """vp_set_batch_tile: fix the batched far sum's tile for a density-chunk width (0: autotune)."""
        _check(load().vp_set_batch_tile(self.handle, C.c_int32(width), C.c_int32(targets_per_thread)), self,
               "vp_set_batch_tile")

    def set_far_sym_cap(self, nbytes: int):
        """vp_set_far_sym_cap: bound on the column scratch of the symmetric far sum."""
        _check(load().vp_set_far_sym_cap(self.handle, C.c_int64(int(nbytes))), self, "vp_set_far_sym_cap")

    def close(self):
        if getattr(self, "handle", None):
            load().vp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx, handle, nt, N, nq):
        self.ctx, self.handle, self.nt, self.N, self.nq = ctx, handle, nt, N, nq

    def release(self):
        if self.handle:
            load().vp_mesh_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class NearField:
    def __init__(self, ctx, mesh, handle, M):
        self.ctx, self.mesh, self.handle, self.M = ctx, mesh, handle, M

    def release(self):
        if self.handle:
            load().vp_nf_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def create(device: int = 0) -> Context:
    return Context(device)


def mesh_upload(ctx: Context, vxy, tri, rule: int = VP_RULE_19_D9, stream=None) -> Mesh:
    lib = load()
    vxy = np.ascontiguousarray(vxy, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    h = C.c_void_p()
    rc = lib.vp_mesh_upload(ctx.handle, vxy.ctypes.data_as(C.c_void_p), C.c_int64(len(vxy)),
                            tri.ctypes.data_as(C.c_void_p), C.c_int64(len(tri)), C.c_int32(rule), _stream(stream),
                            C.byref(h))
    _check(rc, ctx, "vp_mesh_upload")
    nt, N, nq = C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib.vp_mesh_info(h, C.byref(nt), C.byref(N), C.byref(nq)), ctx, "vp_mesh_info")
    return Mesh(ctx, h, nt.value, N.value, nq.value)


def mesh_upload_dev(ctx: Context, vxy_dev, tri_dev, rule: int = VP_RULE_19_D9, stream=None) -> Mesh:
    """vp_mesh_upload_dev: vertices [nv][2] float64 and triangles [nt][3] int32 already on the device."""
    lib = load()
    h = C.c_void_p()
    rc = lib.vp_mesh_upload_dev(ctx.handle, _dptr(vxy_dev, "float64"), C.c_int64(vxy_dev.shape[0]),
                                _dptr(tri_dev, "int32"), C.c_int64(tri_dev.shape[0]), C.c_int32(rule),
                                _stream(stream), C.byref(h))
    _check(rc, ctx, "vp_mesh_upload_dev")
    nt, N, nq = C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib.vp_mesh_info(h, C.byref(nt), C.byref(N), C.byref(nq)), ctx, "vp_mesh_info")
    return Mesh(ctx, h, nt.value, N.value, nq.value)


def mesh_upload_curved(ctx: Context, vxy, tri, curves, rule: int = VP_RULE_19_D9, stream=None) -> Mesh:
    """vp_mesh_upload_curved: host vertices, triangles and curves
    {"cidx": [nt] int32 (-1 straight), "coef": [ncurve][2][K+1] float64}."""
    lib = load()
    vxy = np.ascontiguousarray(vxy, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    cidx = np.ascontiguousarray(curves["cidx"], np.int32)
    coef = np.ascontiguousarray(curves["coef"], np.float64)
    if coef.ndim != 3 or coef.shape[1] != 2 or len(cidx) != len(tri):
        raise ValueError("curves: cidx [nt] and coef [ncurve][2][K+1] expected")
    h = C.c_void_p()
    rc = lib.vp_mesh_upload_curved(ctx.handle, vxy.ctypes.data_as(C.c_void_p), C.c_int64(len(vxy)),
                                   tri.ctypes.data_as(C.c_void_p), C.c_int64(len(tri)),
                                   cidx.ctypes.data_as(C.c_void_p), coef.ctypes.data_as(C.c_void_p),
                                   C.c_int64(coef.shape[0]), C.c_int32(coef.shape[2] - 1), C.c_int32(rule),
                                   _stream(stream), C.byref(h))
    _check(rc, ctx, "vp_mesh_upload_curved")
    nt, N, nq = C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib.vp_mesh_info(h, C.byref(nt), C.byref(N), C.byref(nq)), ctx, "vp_mesh_info")
    return Mesh(ctx, h, nt.value, N.value, nq.value)


class Interp:
    """vp_interp: interpolation of the potential over the elements of a mesh
    (Section 3.5).  curves: None (straight) or {"cidx", "coef"} as for
    mesh_upload_curved."""

    def __init__(self, ctx: Context, vxy, tri, order: int, curves=None, stream=None):
        lib = load()
        self.ctx = ctx
        vxy = np.ascontiguousarray(vxy, np.float64)
        tri = np.ascontiguousarray(tri, np.int32)
        h = C.c_void_p()
        if curves is None:
            rc = lib.vp_interp_create(ctx.handle, vxy.ctypes.data_as(C.c_void_p), C.c_int64(len(vxy)),
                                      tri.ctypes.data_as(C.c_void_p), C.c_int64(len(tri)), None, None,
                                      C.c_int64(0), C.c_int32(0), C.c_int32(order), _stream(stream), C.byref(h))
        else:
            cidx = np.ascontiguousarray(curves["cidx"], np.int32)
            coef = np.ascontiguousarray(curves["coef"], np.float64)
            rc = lib.vp_interp_create(ctx.handle, vxy.ctypes.data_as(C.c_void_p), C.c_int64(len(vxy)),
                                      tri.ctypes.data_as(C.c_void_p), C.c_int64(len(tri)),
                                      cidx.ctypes.data_as(C.c_void_p), coef.ctypes.data_as(C.c_void_p),
                                      C.c_int64(coef.shape[0]), C.c_int32(coef.shape[2] - 1), C.c_int32(order),
                                      _stream(stream), C.byref(h))
        _check(rc, ctx, "vp_interp_create")
        self.handle = h
        nt, n, nn = C.c_int64(), C.c_int64(), C.c_int32()
        _check(lib.vp_interp_info(h, C.byref(nt), C.byref(n), C.byref(nn)), ctx, "vp_interp_info")
        self.nt, self.n_nodes, self.nn, self.order = nt.value, n.value, nn.value, order

    def nodes(self, stream=None):
        import torch
        out = torch.empty((self.n_nodes, 2), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        _check(load().vp_interp_nodes(self.handle, _dptr(out, "float64"), _stream(stream)), self.ctx,
               "vp_interp_nodes")
        return out

    def coeffs(self, u, stream=None):
        """u: device [d][n_nodes] -> device [d][nt][nn]."""
        import torch
        if u.dim() == 1:
            u = u[None, :]
        u = u.contiguous()
        d = u.shape[0]
        out = torch.empty((d, self.nt, self.nn), dtype=torch.float64, device=u.device)
        _check(load().vp_interp_coeffs(self.handle, _dptr(u, "float64"), C.c_int32(d), _dptr(out, "float64"),
                                       _stream(stream)), self.ctx, "vp_interp_coeffs")
        return out

    def eval(self, coef, pts, stream=None):
        """coef [d][nt][nn], pts device [m][2] -> (device [d][m], device [m] int32)."""
        import torch
        coef = coef.contiguous()
        pts = pts.contiguous()
        d, m = coef.shape[0], pts.shape[0]
        out = torch.empty((d, m), dtype=torch.float64, device=pts.device)
        elem = torch.empty(m, dtype=torch.int32, device=pts.device)
        _check(load().vp_interp_eval(self.handle, _dptr(coef, "float64"), C.c_int32(d), _dptr(pts, "float64"),
                                     C.c_int64(m), _dptr(out, "float64"), _dptr(elem, "int32"), _stream(stream)),
               self.ctx, "vp_interp_eval")
        return out, elem

    def release(self):
        if getattr(self, "handle", None):
            load().vp_interp_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def profile_enable(ctx: Context, on: bool = True):
    _check(load().vp_profile_enable(ctx.handle, 1 if on else 0), ctx, "vp_profile_enable")


def profile_reset(ctx: Context):
    _check(load().vp_profile_reset(ctx.handle), ctx, "vp_profile_reset")


def profile_read(ctx: Context) -> dict:
    """{stage: (launches timed, summed device ms)} from the library's CUDA events."""
    cap = 64
    names = C.create_string_buffer(32 * cap)
    counts = np.zeros(cap, np.int64)
    ms = np.zeros(cap, np.float64)
    n = C.c_int32()
    _check(load().vp_profile_read(ctx.handle, names, counts.ctypes.data_as(C.c_void_p), ms.ctypes.data_as(C.c_void_p),
                                  cap, C.byref(n)), ctx, "vp_profile_read")
    out = {}
    for i in range(min(n.value, cap)):
        name = names.raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out[name] = (int(counts[i]), float(ms[i]))
    return out


def mesh_nodes(mesh: Mesh, stream=None):
    import torch
    y = torch.empty((mesh.N, 2), dtype=torch.float64, device=f"cuda:{mesh.ctx.device}")
    w = torch.empty((mesh.N,), dtype=torch.float64, device=f"cuda:{mesh.ctx.device}")
    _check(load().vp_mesh_nodes(mesh.handle, _dptr(y, "float64"), _dptr(w, "float64"), _stream(stream)), mesh.ctx,
           "vp_mesh_nodes")
    return y, w


VP_NF_FP64_WEIGHTS = 1


def nf_params_default() -> dict:
    """vp_nf_params_default: the parameters vp_nearfield_build uses when none are given."""
    p = NfParams()
    _check(load().vp_nf_params_default(C.byref(p)), None, "vp_nf_params_default")
    return {k: getattr(p, k) for k, _ in NfParams._fields_}


def nearfield_build(ctx: Context, mesh: Mesh, node_targets: bool = True, txy=None, eps: float | None = None,
                    c_far: float | None = None, c_near: float | None = None, depth_cap: int | None = None,
                    fp64_weights: bool = False, stream=None) -> NearField:
    """vp_nearfield_build; parameters left as None take the library defaults
    (vp_nf_params_default); fp64_weights sets VP_NF_FP64_WEIGHTS (node
    quadratures in FP64 instead of float-float)."""
    lib = load()
    m = 0 if txy is None else int(txy.shape[0])
    p = NfParams()
    _check(lib.vp_nf_params_default(C.byref(p)), ctx, "vp_nf_params_default")
    if eps is not None:
        p.eps = eps
    if c_far is not None:
        p.c_far = c_far
    if c_near is not None:
        p.c_near = c_near
    if depth_cap is not None:
        p.depth_cap = depth_cap
    p.flags = VP_NF_FP64_WEIGHTS if fp64_weights else 0
    h = C.c_void_p()
    rc = lib.vp_nearfield_build(ctx.handle, mesh.handle, C.c_int32(1 if node_targets else 0),
                                _dptr(txy, "float64") if m else None, C.c_int64(m), C.byref(p), _stream(stream),
                                C.byref(h))
    _check(rc, ctx, "vp_nearfield_build")
    M = (mesh.N if node_targets else 0) + m
    return NearField(ctx, mesh, h, M)


def nearfield_build_host(ctx: Context, mesh: Mesh, node_targets: bool = True, txy: np.ndarray | None = None,
                         fp64_weights: bool = False, stream=None) -> NearField:
    """vp_nearfield_build_host: extra targets from a host array [m][2] (default parameters)."""
    lib = load()
    m = 0 if txy is None else int(txy.shape[0])
    if m:
        txy = np.ascontiguousarray(txy, dtype=np.float64)
    p = NfParams()
    _check(lib.vp_nf_params_default(C.byref(p)), ctx, "vp_nf_params_default")
    p.flags = VP_NF_FP64_WEIGHTS if fp64_weights else 0
    h = C.c_void_p()
    rc = lib.vp_nearfield_build_host(ctx.handle, mesh.handle, C.c_int32(1 if node_targets else 0),
                                     txy.ctypes.data_as(C.c_void_p) if m else None, C.c_int64(m), C.byref(p),
                                     _stream(stream), C.byref(h))
    _check(rc, ctx, "vp_nearfield_build_host")
    M = (mesh.N if node_targets else 0) + m
    return NearField(ctx, mesh, h, M)


def nf_stats(nf: NearField) -> dict:
    s = NfStats()
    _check(load().vp_nf_stats(nf.handle, C.byref(s)), nf.ctx, "vp_nf_stats")
    return s.as_dict()


def nf_prepare_tc(nf: NearField, levels: int = 5, stream=None):
    """vp_nf_prepare_tc: build the tensor-core apply plan (levels 3, 4 or 5)."""
    _check(load().vp_nf_prepare_tc(nf.ctx.handle, nf.handle, C.c_int32(levels), _stream(stream)), nf.ctx,
           "vp_nf_prepare_tc")


def nf_tc_info(nf: NearField) -> dict:
    lv = C.c_int32()
    nt, nc, nb = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().vp_nf_tc_info(nf.handle, C.byref(lv), C.byref(nt), C.byref(nc), C.byref(nb)), nf.ctx,
           "vp_nf_tc_info")
    return {"levels": lv.value, "n_tiles": nt.value, "n_chunks": nc.value, "bytes": nb.value}


def nf_fmm_info(nf: NearField) -> dict:
    lvl, nb = C.c_int32(), C.c_int64()
    _check(load().vp_nf_fmm_info(nf.handle, C.byref(lvl), C.byref(nb)), nf.ctx, "vp_nf_fmm_info")
    return {"leaf_level": lvl.value, "boxes": nb.value}


def device_status(ctx: Context, stream=None) -> int:
    """vp_device_status: synchronise and return (and clear) the device error status."""
    return int(load().vp_device_status(ctx.handle, _stream(stream)))


def nf_lists(nf: NearField, stream=None):
    import torch
    st = nf_stats(nf)
    dev = f"cuda:{nf.ctx.device}"
    row = torch.empty(nf.M + 1, dtype=torch.int64, device=dev)
    tri = torch.empty(max(1, st["n_pairs"]), dtype=torch.int32, device=dev)
    kind = torch.empty(max(1, st["n_pairs"]), dtype=torch.uint8, device=dev)
    tself = torch.empty(nf.M, dtype=torch.int32, device=dev)
    _check(load().vp_nf_lists(nf.handle, _dptr(row, "int64"), _dptr(tri, "int32"), _dptr(kind, "uint8"),
                              _dptr(tself, "int32"), _stream(stream)), nf.ctx, "vp_nf_lists")
    P = st["n_pairs"]
    return row, tri[:P], kind[:P], tself


def nf_weights(nf: NearField, stream=None):
    import torch
    P = nf_stats(nf)["n_pairs"]
    w = torch.empty((max(1, P), nf.mesh.nq), dtype=torch.float64, device=f"cuda:{nf.ctx.device}")
    _check(load().vp_nf_weights(nf.handle, _dptr(w, "float64"), _stream(stream)), nf.ctx, "vp_nf_weights")
    return w[:P]


def potential_eval(ctx: Context, nf: NearField, f, precision: int = VP_FP64, out=None, stream=None):
    """u [d][M] on the device for densities f [d][N] (CUDA float64)."""
    import torch
    if f.dim() == 1:
        f = f.unsqueeze(0)
    d = int(f.shape[0])
    if f.shape[1] != nf.mesh.N:
        raise ValueError("f must be [d][N]")
    if out is None:
        out = torch.empty((d, nf.M), dtype=torch.float64, device=f.device)
    rc = load().vp_potential_eval(ctx.handle, nf.handle, _dptr(f, "float64"), C.c_int32(d), _dptr(out, "float64"),
                                  C.c_int32(precision), _stream(stream))
    _check(rc, ctx, "vp_potential_eval")
    return out


def potential_eval_noalloc(ctx: Context, nf: NearField, f, precision: int = VP_FP64, out=None, stream=None):
    """vp_potential_eval_noalloc: like potential_eval, with the library's fixed
    scratch instead of allocated memory (for callers that cannot allocate
    device memory while they evaluate).  `out` must be given if the caller
    cannot allocate either."""
    import torch
    if f.dim() == 1:
        f = f.unsqueeze(0)
    d = int(f.shape[0])
    if f.shape[1] != nf.mesh.N:
        raise ValueError("f must be [d][N]")
    if out is None:
        out = torch.empty((d, nf.M), dtype=torch.float64, device=f.device)
    rc = load().vp_potential_eval_noalloc(ctx.handle, nf.handle, _dptr(f, "float64"), C.c_int32(d),
                                          _dptr(out, "float64"), C.c_int32(precision), _stream(stream))
    _check(rc, ctx, "vp_potential_eval_noalloc")
    return out


def potential_eval_host(ctx: Context, nf: NearField, f_host: np.ndarray, precision: int = VP_FP64, out=None,
                        stream=None):
    """Same as potential_eval with host buffers (numpy or pinned CPU tensors)."""
    f_host = f_host if not isinstance(f_host, np.ndarray) else np.ascontiguousarray(np.atleast_2d(f_host), np.float64)
    d = int(f_host.shape[0])
    if out is None:
        out = np.empty((d, nf.M), dtype=np.float64)
    fp = f_host.ctypes.data_as(C.c_void_p) if isinstance(f_host, np.ndarray) else C.c_void_p(f_host.data_ptr())
    up = out.ctypes.data_as(C.c_void_p) if isinstance(out, np.ndarray) else C.c_void_p(out.data_ptr())
    rc = load().vp_potential_eval_host(ctx.handle, nf.handle, fp, C.c_int32(d), up, C.c_int32(precision),
                                       _stream(stream))
    _check(rc, ctx, "vp_potential_eval_host")
    return out


def potential_eval_batch(ctx: Context, items, precision: int = VP_FP64, stream=None):
    """items: list of (nf, f [d][N] cuda, u [d][M] cuda)."""
    arr = (EvalItem * len(items))()
    for i, (nf, f, u) in enumerate(items):
        arr[i].nf = nf.handle
        arr[i].f_dev = f.data_ptr()
        arr[i].d = int(f.shape[0])
        arr[i].u_dev = u.data_ptr()
    rc = load().vp_potential_eval_batch(ctx.handle, arr, C.c_int32(len(items)), C.c_int32(precision), _stream(stream))
    _check(rc, ctx, "vp_potential_eval_batch")


class Batch:
    """A prepared, graph-captured batch (vp_batch_create / vp_batch_launch)."""

    def __init__(self, ctx: Context, items, precision: int = VP_MIXED, stream=None):
        self.ctx = ctx
        self.items = list(items)         # keep the tensors alive
        arr = (EvalItem * len(self.items))()
        for i, (nf, f, u) in enumerate(self.items):
            arr[i].nf = nf.handle
            arr[i].f_dev = f.data_ptr()
            arr[i].d = int(f.shape[0])
            arr[i].u_dev = u.data_ptr()
        h = C.c_void_p()
        _check(load().vp_batch_create(ctx.handle, arr, C.c_int32(len(self.items)), C.c_int32(precision),
                                      _stream(stream), C.byref(h)), ctx, "vp_batch_create")
        self.handle = h

    def launch(self, stream=None):
        _check(load().vp_batch_launch(self.handle, _stream(stream)), self.ctx, "vp_batch_launch")

    def info(self) -> dict:
        """vp_batch_info: targets-per-thread tile and work units per density-chunk width (1, 2, 4, 8)."""
        tpt = (C.c_int32 * 4)()
        units = (C.c_int64 * 4)()
        _check(load().vp_batch_info(self.handle, tpt, units), self.ctx, "vp_batch_info")
        return {w: (tpt[i], units[i]) for i, w in enumerate((1, 2, 4, 8))}

    def release(self):
        if getattr(self, "handle", None):
            load().vp_batch_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Server:
    """vp_server_*: continuous-batching serving loop over resident meshes."""

    def __init__(self, ctx: Context, slots: int = 4, hbm_budget_bytes: int = 8 << 30, precision: int = VP_MIXED):
        self.ctx = ctx
        h = C.c_void_p()
        _check(load().vp_server_create(ctx.handle, C.c_int32(slots), C.c_int64(hbm_budget_bytes),
                                       C.c_int32(precision), C.byref(h)), ctx, "vp_server_create")
        self.handle = h
        self._keep = {}

    def register(self, key: int, nf: NearField):
        _check(load().vp_server_register(self.handle, C.c_int64(key), nf.handle), self.ctx, "vp_server_register")
        self._keep[("nf", key)] = nf

    def register_cold(self, key: int, vxy, tri, rule: int = VP_RULE_19_D9):
        vxy = np.ascontiguousarray(vxy, np.float64)
        tri = np.ascontiguousarray(tri, np.int32)
        _check(load().vp_server_register_cold(self.handle, C.c_int64(key), vxy.ctypes.data_as(C.c_void_p),
                                              C.c_int64(len(vxy)), tri.ctypes.data_as(C.c_void_p),
                                              C.c_int64(len(tri)), C.c_int32(rule)), self.ctx,
               "vp_server_register_cold")

    def mesh_size(self, key: int):
        n, m = C.c_int64(), C.c_int64()
        _check(load().vp_server_mesh_size(self.handle, C.c_int64(key), C.byref(n), C.byref(m)), self.ctx,
               "vp_server_mesh_size")
        return n.value, m.value

    def submit(self, key: int, f_host: np.ndarray, u_host: np.ndarray) -> int:
        """f_host [d][N], u_host [d][M]: contiguous float64 host arrays kept
        alive by the caller until the request completes."""
        if f_host.dtype != np.float64 or u_host.dtype != np.float64 or not f_host.flags.c_contiguous \
                or not u_host.flags.c_contiguous:
            raise TypeError("f_host and u_host must be contiguous float64 arrays")
        t = C.c_int64()
        _check(load().vp_server_submit(self.handle, C.c_int64(key), f_host.ctypes.data_as(C.c_void_p),
                                       C.c_int32(f_host.shape[0]), u_host.ctypes.data_as(C.c_void_p), C.byref(t)),
               self.ctx, "vp_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_s: float = 600.0):
        st, lat = C.c_int32(), C.c_double()
        _check(load().vp_server_wait(self.handle, C.c_int64(ticket), C.c_double(timeout_s), C.byref(st),
                                     C.byref(lat)), self.ctx, "vp_server_wait")
        return st.value, lat.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().vp_server_stats(self.handle, C.byref(s)), self.ctx, "vp_server_stats")
        return s.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            load().vp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pinned_empty(shape):
    """A page-locked host float64 array (numpy view of a pinned torch tensor)."""
    import torch
    return torch.empty(shape, dtype=torch.float64).pin_memory().numpy()


def far_rule(rule: int):
    """(x, y, w, what, degree) of a far rule: VP_RULE_16_D8, VP_RULE_19_D9, VP_RULE_CONICAL(n) or
    VP_RULE_SYM(n)."""
    lib = load()
    n = C.c_int32()
    what = C.c_double()
    deg = C.c_int32()
    _check(lib.vp_far_rule(rule, None, None, None, C.byref(what), C.byref(deg), 0, C.byref(n)), None, "vp_far_rule")
    k = n.value
    x, y, w = (np.zeros(k) for _ in range(3))
    _check(lib.vp_far_rule(rule, x.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p),
                           w.ctypes.data_as(C.c_void_p), C.byref(what), C.byref(deg), k, C.byref(n)), None,
           "vp_far_rule")
    return x, y, w, what.value, deg.value


def rule_table(which: int):
    """(x, y, w, what) of a compiled rule: 16, 19 (far), 33 (near), 8 (radial GGQ), 5 (radial rule of the
    float-float self weights: w for int r p, y for int r log(r) p), 116 (arc-length)."""
    lib = load()
    cap = 64
    x, y, w = (np.zeros(cap) for _ in range(3))
    what = C.c_double()
    n = C.c_int32()
    _check(lib.vp_rule_table(which, x.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p),
                             w.ctypes.data_as(C.c_void_p), C.byref(what), cap, C.byref(n)), None, "vp_rule_table")
    k = n.value
    return x[:k].copy(), y[:k].copy(), w[:k].copy(), what.value
