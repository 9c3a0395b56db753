"""Python binding of libpermanova (PERMANOVA's s_W on GB300, sm_103a).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libpermanova.so``; tensors are passed as raw device pointers
(``torch.Tensor.data_ptr()``) and streams as ``cudaStream_t`` handles.  The
functions carry the C ABI's names (``include/permanova.h``) and raise
:class:`PermanovaError` on a non-zero status.  There is no CPU fallback: if
the library has not been built (``paper_2505_04556_gb300.build()``),
loading it fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpermanova.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "permanova.h")

# permanova_status
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
# permanova_label_t
LABEL_I32, LABEL_U16, LABEL_U8 = 0, 1, 2
# permanova_form_t
FORM_AUTO, FORM_BRUTE, FORM_PERMBLOCK, FORM_GEMM = 0, 1, 2, 3
FORM_NAMES = {FORM_AUTO: "auto", FORM_BRUTE: "brute", FORM_PERMBLOCK: "permblock", FORM_GEMM: "gemm"}

_STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA",
                 ETIMEOUT: "ETIMEOUT", EUNSUPPORTED: "EUNSUPPORTED"}


class PermanovaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class permanova_result(ctypes.Structure):
    _fields_ = [("s_T", ctypes.c_double), ("s_W_obs", ctypes.c_double),
                ("F_obs", ctypes.c_double), ("p_value", ctypes.c_double),
                ("n_ge", ctypes.c_uint64), ("n_perms", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class permanova_plan_t(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("permblock_variant", ctypes.c_int),
                ("gemm_rows_div", ctypes.c_uint32), ("gemm_drain_kblocks", ctypes.c_uint32),
                ("brute_chunk_mult", ctypes.c_uint32)]


class permanova_profile_t(ctypes.Structure):
    _fields_ = [("main_kernel_ms", ctypes.c_double), ("main_kernel_launches", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("last_form", ctypes.c_int),
                ("host_calls", ctypes.c_uint64), ("host_total_ms", ctypes.c_double),
                ("host_first_segment_ms", ctypes.c_double), ("host_copy_ms", ctypes.c_double),
                ("host_h2d_bytes", ctypes.c_uint64), ("host_segments", ctypes.c_uint32),
                ("host_seg_landed_ms", ctypes.c_double * 16), ("host_seg_done_ms", ctypes.c_double * 16)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        m = min(16, d["host_segments"])
        d["host_seg_landed_ms"] = list(d["host_seg_landed_ms"])[:m]
        d["host_seg_done_ms"] = list(d["host_seg_done_ms"])[:m]
        return d


_lock = threading.Lock()
_lib = None


def exported_names() -> list[str]:
    """Function names declared in include/permanova.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|size_t|const char \*)\s*\*?\s*(permanova_\w+)\s*\(",
                                 txt, re.M)))


def load(path: str | None = None):
    """Load libpermanova.so and declare its signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} is missing: build it with paper_2505_04556_gb300.build() "
                              "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        vp, u32, u64, i32, sz = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                 ctypes.c_size_t)
        lib.permanova_create.argtypes = [i32, sz, ctypes.POINTER(vp)]
        lib.permanova_create.restype = i32
        lib.permanova_destroy.argtypes = [vp]
        lib.permanova_destroy.restype = None
        lib.permanova_last_error.argtypes = [vp]
        lib.permanova_last_error.restype = ctypes.c_char_p
        lib.permanova_set_form.argtypes = [vp, i32]
        lib.permanova_set_form.restype = i32
        lib.permanova_plan_form.argtypes = [vp, u32, u32, u64]
        lib.permanova_plan_form.restype = i32
        lib.permanova_set_plan.argtypes = [vp, ctypes.POINTER(permanova_plan_t)]
        lib.permanova_set_plan.restype = i32
        lib.permanova_plan_describe.argtypes = [vp, u32, u32, u64, ctypes.c_char_p, sz]
        lib.permanova_plan_describe.restype = i32
        lib.permanova_scratch_bytes.argtypes = [vp, i32, u32, u32, u64]
        lib.permanova_scratch_bytes.restype = sz
        lib.permanova_scratch_reserved.argtypes = [vp]
        lib.permanova_scratch_reserved.restype = sz
        lib.permanova_reserve_scratch.argtypes = [vp, sz]
        lib.permanova_reserve_scratch.restype = i32
        lib.permanova_release_scratch.argtypes = [vp]
        lib.permanova_release_scratch.restype = i32
        sw_args = [vp, vp, u32, u64, vp, i32, u32, u64, vp, vp, vp]
        lib.permanova_sW.argtypes = sw_args
        lib.permanova_sW.restype = i32
        lib.permanova_sW_host.argtypes = sw_args
        lib.permanova_sW_host.restype = i32
        lib.permanova_sync.argtypes = [vp, vp]
        lib.permanova_sync.restype = i32
        lib.permanova_permutations.argtypes = [vp, vp, u32, u32, u64, u64, vp, i32, vp]
        lib.permanova_permutations.restype = i32
        lib.permanova_test.argtypes = [vp, vp, u32, u64, vp, u32, u64, u64,
                                       ctypes.POINTER(permanova_result), vp, vp]
        lib.permanova_test.restype = i32
        lib.permanova_autotune.argtypes = [vp, vp, u32, u64, vp, i32, u32, u64, vp,
                                           ctypes.POINTER(i32), vp]
        lib.permanova_autotune.restype = i32
        lib.permanova_test_batch.argtypes = [vp, vp, u32, u64, vp, u32, u32, u64, vp,
                                             ctypes.POINTER(permanova_result), vp, vp]
        lib.permanova_test_batch.restype = i32
        lib.permanova_test_mixed.argtypes = [vp, vp, u32, u64, vp, u32, vp, vp, vp,
                                             ctypes.POINTER(permanova_result), vp, vp]
        lib.permanova_test_mixed.restype = i32
        lib.permanova_prepare.argtypes = [vp, vp, u32, u64, ctypes.POINTER(vp), vp]
        lib.permanova_prepare.restype = i32
        lib.permanova_prepared_destroy.argtypes = [vp]
        lib.permanova_prepared_destroy.restype = None
        lib.permanova_sW_prepared.argtypes = [vp, vp, vp, i32, u32, u64, vp, vp, vp]
        lib.permanova_sW_prepared.restype = i32
        lib.permanova_test_mixed_prepared.argtypes = [vp, vp, vp, u32, vp, vp, vp,
                                                      ctypes.POINTER(permanova_result), vp, vp]
        lib.permanova_test_mixed_prepared.restype = i32
        lib.permanova_selftest_wait.argtypes = [vp, u32, vp]
        lib.permanova_selftest_wait.restype = i32
        lib.permanova_set_graphs.argtypes = [vp, i32]
        lib.permanova_set_graphs.restype = i32
        lib.permanova_sW_noalloc.argtypes = [vp, u32, u64, vp, i32, u32, u64, vp, vp, vp]
        lib.permanova_sW_noalloc.restype = i32
        lib.permanova_profile_enable.argtypes = [vp, i32]
        lib.permanova_profile_enable.restype = i32
        lib.permanova_profile_read.argtypes = [vp, ctypes.POINTER(permanova_profile_t)]
        lib.permanova_profile_read.restype = i32
        _lib = lib
        return lib


def build(force: bool = False) -> str:
    from . import native_build
    return native_build.build(force=force)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _check(ctx, rc: int):
    if rc != OK:
        msg = load().permanova_last_error(ctx)
        raise PermanovaError(rc, msg.decode() if msg else "")


def _ptr(x):
    """Raw address of a torch tensor, numpy array or integer (0/None = NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def label_type_of(t) -> int:
    """Label type code of a torch tensor / numpy array of labels."""
    name = str(t.dtype).replace("torch.", "")
    return {"uint8": LABEL_U8, "uint16": LABEL_U16, "int16": LABEL_U16, "int32": LABEL_I32}[name]


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------

def permanova_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = ctypes.c_void_p()
    rc = load().permanova_create(int(device), int(hbm_budget_bytes), ctypes.byref(h))
    _check(None, rc)
    return h.value


def permanova_destroy(ctx) -> None:
    load().permanova_destroy(ctx)


def permanova_last_error(ctx) -> str:
    return load().permanova_last_error(ctx).decode()


def permanova_set_form(ctx, form: int) -> None:
    _check(ctx, load().permanova_set_form(ctx, int(form)))


def permanova_plan_form(ctx, n_dims: int, n_groups: int, n_perms: int) -> int:
    return int(load().permanova_plan_form(ctx, n_dims, n_groups, n_perms))


def permanova_set_plan(ctx, form: int, permblock_variant: int = 0, gemm_rows_div: int = 0,
                       gemm_drain_kblocks: int = 0, brute_chunk_mult: int = 0) -> None:
    pl = permanova_plan_t(int(form), int(permblock_variant), int(gemm_rows_div),
                          int(gemm_drain_kblocks), int(brute_chunk_mult))
    _check(ctx, load().permanova_set_plan(ctx, ctypes.byref(pl)))


def permanova_plan_describe(ctx, n_dims: int, n_groups: int, n_perms: int) -> dict:
    import json
    buf = ctypes.create_string_buffer(512)
    _check(ctx, load().permanova_plan_describe(ctx, int(n_dims), int(n_groups), int(n_perms), buf, 512))
    return json.loads(buf.value.decode())


def permanova_scratch_bytes(ctx, form: int, n_dims: int, n_groups: int, n_perms: int) -> int:
    return int(load().permanova_scratch_bytes(ctx, int(form), n_dims, n_groups, n_perms))


def permanova_scratch_reserved(ctx) -> int:
    return int(load().permanova_scratch_reserved(ctx))


def permanova_reserve_scratch(ctx, nbytes: int) -> None:
    _check(ctx, load().permanova_reserve_scratch(ctx, int(nbytes)))


def permanova_release_scratch(ctx) -> None:
    _check(ctx, load().permanova_release_scratch(ctx))


def permanova_sW(ctx, mat, n_dims: int, ld: int, groupings, label_type: int, n_groups: int,
                 n_perms: int, inv_group_sizes, out_sW, stream=None) -> None:
    rc = load().permanova_sW(ctx, _ptr(mat), int(n_dims), int(ld), _ptr(groupings), int(label_type),
                             int(n_groups), int(n_perms), _ptr(inv_group_sizes), _ptr(out_sW),
                             _stream(stream))
    _check(ctx, rc)


def permanova_sW_host(ctx, mat, n_dims: int, ld: int, groupings, label_type: int, n_groups: int,
                      n_perms: int, inv_group_sizes, out_sW, stream=None) -> None:
    rc = load().permanova_sW_host(ctx, _ptr(mat), int(n_dims), int(ld), _ptr(groupings),
                                  int(label_type), int(n_groups), int(n_perms),
                                  _ptr(inv_group_sizes), _ptr(out_sW), _stream(stream))
    _check(ctx, rc)


def permanova_autotune(ctx, mat, n_dims: int, ld: int, groupings, label_type: int, n_groups: int,
                       n_perms: int, inv_group_sizes, stream=None) -> int:
    form = ctypes.c_int(0)
    rc = load().permanova_autotune(ctx, _ptr(mat), int(n_dims), int(ld), _ptr(groupings),
                                   int(label_type), int(n_groups), int(n_perms),
                                   _ptr(inv_group_sizes), ctypes.byref(form), _stream(stream))
    _check(ctx, rc)
    return form.value


def permanova_test_batch(ctx, mat, n_dims: int, ld: int, groupings, n_tests: int, n_groups: int,
                         n_perms: int, seeds, out_sW=None, stream=None) -> list:
    res = (permanova_result * n_tests)()
    sd = (ctypes.c_uint64 * n_tests)(*[int(x) & (2**64 - 1) for x in seeds])
    rc = load().permanova_test_batch(ctx, _ptr(mat), int(n_dims), int(ld), _ptr(groupings),
                                     int(n_tests), int(n_groups), int(n_perms),
                                     ctypes.cast(sd, ctypes.c_void_p), res, _ptr(out_sW),
                                     _stream(stream))
    _check(ctx, rc)
    return [r.as_dict() for r in res]


def permanova_test_mixed(ctx, mat, n_dims: int, ld: int, groupings, n_groups, n_perms, seeds,
                         out_sW=None, stream=None) -> list:
    T = len(seeds)
    res = (permanova_result * T)()
    ks = (ctypes.c_uint32 * T)(*[int(k) for k in n_groups])
    ps = (ctypes.c_uint64 * T)(*[int(p) for p in n_perms])
    sd = (ctypes.c_uint64 * T)(*[int(x) & (2**64 - 1) for x in seeds])
    rc = load().permanova_test_mixed(ctx, _ptr(mat), int(n_dims), int(ld), _ptr(groupings), T,
                                     ctypes.cast(ks, ctypes.c_void_p), ctypes.cast(ps, ctypes.c_void_p),
                                     ctypes.cast(sd, ctypes.c_void_p), res, _ptr(out_sW),
                                     _stream(stream))
    _check(ctx, rc)
    return [r.as_dict() for r in res]


def permanova_prepare(ctx, mat, n_dims: int, ld: int, stream=None):
    h = ctypes.c_void_p()
    rc = load().permanova_prepare(ctx, _ptr(mat), int(n_dims), int(ld), ctypes.byref(h), _stream(stream))
    _check(ctx, rc)
    return h.value


def permanova_prepared_destroy(prepared) -> None:
    load().permanova_prepared_destroy(prepared)


def permanova_sW_prepared(ctx, prepared, groupings, label_type: int, n_groups: int, n_perms: int,
                          inv_group_sizes, out_sW, stream=None) -> None:
    rc = load().permanova_sW_prepared(ctx, prepared, _ptr(groupings), int(label_type), int(n_groups),
                                      int(n_perms), _ptr(inv_group_sizes), _ptr(out_sW), _stream(stream))
    _check(ctx, rc)


def permanova_test_mixed_prepared(ctx, prepared, groupings, n_groups, n_perms, seeds, out_sW=None,
                                  stream=None) -> list:
    T = len(seeds)
    res = (permanova_result * T)()
    ks = (ctypes.c_uint32 * T)(*[int(k) for k in n_groups])
    ps = (ctypes.c_uint64 * T)(*[int(p) for p in n_perms])
    sd = (ctypes.c_uint64 * T)(*[int(x) & (2**64 - 1) for x in seeds])
    rc = load().permanova_test_mixed_prepared(ctx, prepared, _ptr(groupings), T,
                                              ctypes.cast(ks, ctypes.c_void_p),
                                              ctypes.cast(ps, ctypes.c_void_p),
                                              ctypes.cast(sd, ctypes.c_void_p), res, _ptr(out_sW),
                                              _stream(stream))
    _check(ctx, rc)
    return [r.as_dict() for r in res]


def permanova_selftest_wait(ctx, limit_us: int, stream=None) -> None:
    _check(ctx, load().permanova_selftest_wait(ctx, int(limit_us), _stream(stream)))


def permanova_set_graphs(ctx, enable: bool = True) -> None:
    _check(ctx, load().permanova_set_graphs(ctx, 1 if enable else 0))


def permanova_sW_noalloc(mat, n_dims: int, ld: int, groupings, label_type: int, n_groups: int,
                         n_perms: int, inv_group_sizes, out_sW, stream=None) -> None:
    """s_W with no device allocation: the scratch is a fixed 8 MiB array that
    the library keeps resident on the device, for callers that may not call
    cudaMalloc (plugins of frameworks that own all device memory, processes
    in a fixed memory pool).  Synchronises the stream."""
    rc = load().permanova_sW_noalloc(_ptr(mat), int(n_dims), int(ld), _ptr(groupings),
                                     int(label_type), int(n_groups), int(n_perms),
                                     _ptr(inv_group_sizes), _ptr(out_sW), _stream(stream))
    _check(None, rc)


def permanova_sync(ctx, stream=None) -> None:
    _check(ctx, load().permanova_sync(ctx, _stream(stream)))


def permanova_permutations(ctx, grouping, n_dims: int, n_groups: int, n_perms: int, seed: int,
                           out, label_type: int, stream=None) -> None:
    rc = load().permanova_permutations(ctx, _ptr(grouping), int(n_dims), int(n_groups),
                                       int(n_perms), int(seed) & (2**64 - 1), _ptr(out),
                                       int(label_type), _stream(stream))
    _check(ctx, rc)


def permanova_test(ctx, mat, n_dims: int, ld: int, grouping, n_groups: int, n_perms: int,
                   seed: int, out_sW=None, stream=None) -> dict:
    res = permanova_result()
    rc = load().permanova_test(ctx, _ptr(mat), int(n_dims), int(ld), _ptr(grouping),
                               int(n_groups), int(n_perms), int(seed) & (2**64 - 1),
                               ctypes.byref(res), _ptr(out_sW), _stream(stream))
    _check(ctx, rc)
    return res.as_dict()


def permanova_profile_enable(ctx, enable: bool = True) -> None:
    _check(ctx, load().permanova_profile_enable(ctx, 1 if enable else 0))


def permanova_profile_read(ctx) -> dict:
    out = permanova_profile_t()
    _check(ctx, load().permanova_profile_read(ctx, ctypes.byref(out)))
    return out.as_dict()


class Context:
    """Owns one permanova_ctx; a convenience around the functions above."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.handle = permanova_create(device, hbm_budget_bytes)

    def close(self):
        if self.handle:
            permanova_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_form(self, form: int):
        permanova_set_form(self.handle, form)

    def sW(self, mat, groupings, n_groups: int, inv_group_sizes, out=None, stream=None):
        """s_W for every row of ``groupings`` (P x n torch tensor on the GPU)."""
        import torch
        n = mat.shape[0]
        P = groupings.shape[0]
        if out is None:
            out = torch.empty(P, dtype=torch.float64, device=mat.device)
        permanova_sW(self.handle, mat, n, mat.stride(0), groupings, label_type_of(groupings),
                     n_groups, P, inv_group_sizes, out, stream)
        return out

    def test(self, mat, grouping, n_groups: int, n_perms: int, seed: int, out_sW=None,
             stream=None) -> dict:
        return permanova_test(self.handle, mat, mat.shape[0], mat.stride(0), grouping, n_groups,
                              n_perms, seed, out_sW, stream)
