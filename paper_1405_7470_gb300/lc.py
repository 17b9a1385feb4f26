"""Thin ctypes binding of the C ABI declared in include/lc.h.

Argument marshalling only: every step of the contraction runs in the CUDA
library. Torch is used for device memory (``data_ptr``) and streams
(``cuda_stream``). There is no CPU fallback: if ``liblc.so`` is missing or fails
to load, every call raises.

The raw entry points keep the C names (``lc_kernel_create``, ``lc_contract``,
...); ``Kernel``, ``Variant`` and ``contract`` wrap them for torch tensors.
"""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblc.so")

LC_OK = 0
STATUS = {
    0: "LC_OK", 1: "LC_ERR_INVALID_ARGUMENT", 2: "LC_ERR_UNSUPPORTED", 3: "LC_ERR_INVALID_VARIANT",
    4: "LC_ERR_ASSUMPTION", 5: "LC_ERR_MISALIGNED", 6: "LC_ERR_BUFFER_TOO_SMALL", 7: "LC_ERR_CUDA",
    8: "LC_ERR_TIMEOUT", 9: "LC_ERR_NO_DEVICE", 10: "LC_ERR_NOT_FOUND", 11: "LC_ERR_INDEX",
}
ENGINE = {"simt": 0, "tcgen05": 1, "warp": 2, "ksplit": 3}
LAYOUT = {"elem": 0, "node": 1}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2, "bf16x3": 3}
DTYPE_F32, DTYPE_F64 = 0, 1

DOMAIN = "{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }"
INSTRUCTION = "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])"


class LcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class lc_variant(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32)] + [
        (n, ctypes.c_int32) for n in (
            "engine", "layout", "precision", "tile_e", "elems_per_thread", "split_i", "unroll",
            "prefetch_smem", "tail_free", "stages", "ctas_per_sm", "out_buffers", "store_rows", "max_ctas",
            "mma_order", "a_operand")
    ]


class lc_plan(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("grid", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("tiles", ctypes.c_int64)] + [
        (n, ctypes.c_int32) for n in (
            "column_blocks", "ops_per_block", "k_mma", "k_block", "cols_per_op", "mma_n", "stacked", "a_buffers",
            "out_slots", "store_rows", "mma_per_tile", "a_in_tmem", "tmem_cols")
    ]


class lc_group(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int64), ("N", ctypes.c_int32), ("F", ctypes.c_int32),
                ("D_dev", ctypes.c_void_p), ("u_dev", ctypes.c_void_p), ("out_dev", ctypes.c_void_p)]


# Exported symbols and their signatures (argtypes, restype).
_P, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_VP = ctypes.POINTER(lc_variant)
SIGNATURES = {
    "lc_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "lc_last_cuda_error": ([], ctypes.c_int),
    "lc_kernel_create": ([ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(_P)], ctypes.c_int),
    "lc_kernel_destroy": ([_P], None),
    "lc_kernel_print": ([_P, _VP, ctypes.c_char_p, _SZ, ctypes.POINTER(_SZ)], ctypes.c_int),
    "lc_variant_default": ([_P, _I64, _I32, _I32, _I32, _I32, _VP], ctypes.c_int),
    "lc_variant_validate": ([_P, _I64, _I32, _I32, _VP], ctypes.c_int),
    "lc_variant_plan": ([_P, _I64, _I32, _I32, _VP, ctypes.POINTER(lc_plan)], ctypes.c_int),
    "lc_contract": ([_P, _VP, _P, _P, _P, _I64, _I32, _I32, _P], ctypes.c_int),
    "lc_contract_geo": ([_P, _VP, _P, _P, _P, _P, _I64, _I32, _I32, _P], ctypes.c_int),
    "lc_lift": ([_P, _VP, _P, _P, _P, _P, _P, _P, _I64, _I32, _I32, _I32, _I32, _P], ctypes.c_int),
    "lc_kernel_signature": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)], ctypes.c_int),
    "lc_kernel_arg_name": ([_P, _I32, _I32, ctypes.c_char_p, _SZ], ctypes.c_int),
    "lc_elementwise_source": ([_P, _VP, _P, ctypes.c_char_p, _SZ, ctypes.POINTER(_SZ)], ctypes.c_int),
    "lc_elementwise": ([_P, _VP, _P, _P, _P, _P], ctypes.c_int),
    "lc_contract_host": ([_P, _VP, _P, _P, _P, _I64, _I32, _I32, _P, _P, _P, _P], ctypes.c_int),
    "lc_device_error": ([ctypes.c_int], ctypes.c_int),
    "lc_selftest_wait_timeout": ([_I64, _P], ctypes.c_int),
    "lc_error_norm_workspace_size": ([_I64, ctypes.POINTER(_SZ)], ctypes.c_int),
    "lc_error_norm": ([_P, _I32, _P, _I64, _P, _P, _SZ, _P], ctypes.c_int),
    "lc_error_norm_noalloc": ([_P, _I32, _P, _I64, _P, _P], ctypes.c_int),
    "lc_device_info": ([ctypes.POINTER(_I32)] * 3, ctypes.c_int),
    "lc_grouped_workspace_size": ([_P, _VP, ctypes.POINTER(lc_group), _I32, ctypes.POINTER(_SZ)], ctypes.c_int),
    "lc_grouped_plan_create": ([_P, _VP, ctypes.POINTER(lc_group), _I32, _P, _SZ, _I32, _P, ctypes.POINTER(_P)],
                               ctypes.c_int),
    "lc_grouped_run": ([_P, _P], ctypes.c_int),
    "lc_grouped_plan_info": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)], ctypes.c_int),
    "lc_grouped_plan_group": ([_P, _I32, _VP], ctypes.c_int),
    "lc_grouped_plan_destroy": ([_P], None),
    "lc_enumerate_variants": ([_P, _I64, _I32, _I32, _I32, _I32, _VP, _I32, ctypes.POINTER(_I32)], ctypes.c_int),
    "lc_autotune": ([_P, _I64, _I32, _I32, _I32, _I32, _P, _P, _P, _I32, _VP, _P, _I32, ctypes.POINTER(_I32), _P],
                    ctypes.c_int),
    "lc_mlp_param_count": ([_I32, ctypes.POINTER(_I64)], ctypes.c_int),
    "lc_mlp_forward": ([_P, _P, _I64, _I32, _P, _P], ctypes.c_int),
    "lc_mlp_workspace_size": ([_I32, ctypes.POINTER(_SZ)], ctypes.c_int),
    "lc_mlp_loss_grad": ([_P, _P, _P, _I64, _I32, _P, _P, _SZ, _P], ctypes.c_int),
    "lc_mlp_adam_step": ([_P, _P, _P, _P, _I64, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, _P], ctypes.c_int),
    "lc_variant_features": ([_P, _I64, _I32, _I32, _I32, _I32, _VP, _P], ctypes.c_int),
    "lc_pick_workspace_size": ([ctypes.POINTER(_SZ)], ctypes.c_int),
    "lc_pick_variant": ([_P, _I64, _I32, _I32, _I32, _I32, _P, _P, _SZ, _VP, ctypes.POINTER(ctypes.c_float), _P],
                        ctypes.c_int),
    "lc_pick_variant_ensemble": ([_P, _I64, _I32, _I32, _I32, _I32, _P, _I32, _P, _SZ, _VP,
                                  ctypes.POINTER(ctypes.c_float), _P], ctypes.c_int),
}
FEATURES = 32  # LC_FEATURES

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load liblc.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
            lib = ctypes.CDLL(p)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def check(st: int, what: str = "lc"):
    if st != LC_OK:
        raise LcError(st, what)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Kernel:
    """Immutable kernel handle: loop domain + instruction + assumptions (Section 2.1)."""

    def __init__(self, domain: str = DOMAIN, instruction: str = INSTRUCTION, assumptions: str | None = None):
        lib = load()
        h = ctypes.c_void_p()
        st = lib.lc_kernel_create(domain.encode(), instruction.encode(),
                                  assumptions.encode() if assumptions else None, ctypes.byref(h))
        check(st, "lc_kernel_create")
        self._h = h
        self._lib = lib

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lc_kernel_destroy(self._h)
            self._h = None

    def print(self, variant: "lc_variant | None" = None) -> str:
        need = ctypes.c_size_t(0)
        vp = ctypes.byref(variant) if variant is not None else None
        self._lib.lc_kernel_print(self._h, vp, None, 0, ctypes.byref(need))
        buf = ctypes.create_string_buffer(need.value)
        check(self._lib.lc_kernel_print(self._h, vp, buf, need.value, ctypes.byref(need)), "lc_kernel_print")
        return buf.value.decode()


def Variant(engine="simt", layout="elem", precision="fp32", tile_e=64, elems_per_thread=4, split_i=8,
            unroll=4, prefetch_smem=1, tail_free=0, stages=1, ctas_per_sm=0, out_buffers=0,
            store_rows=0, max_ctas=0, mma_order=0, a_operand=0) -> lc_variant:
    v = lc_variant()
    v.struct_size = ctypes.sizeof(lc_variant)
    v.engine = ENGINE[engine] if isinstance(engine, str) else engine
    v.layout = LAYOUT[layout] if isinstance(layout, str) else layout
    v.precision = PRECISION[precision] if isinstance(precision, str) else precision
    v.tile_e, v.elems_per_thread, v.split_i, v.unroll = tile_e, elems_per_thread, split_i, unroll
    v.prefetch_smem, v.tail_free, v.stages, v.ctas_per_sm = prefetch_smem, tail_free, stages, ctas_per_sm
    v.out_buffers, v.store_rows, v.max_ctas = out_buffers, store_rows, max_ctas
    v.mma_order, v.a_operand = mma_order, a_operand
    return v


def variant_dict(v: lc_variant) -> dict:
    inv = lambda m, x: next((k for k, val in m.items() if val == x), x)
    return dict(engine=inv(ENGINE, v.engine), layout=inv(LAYOUT, v.layout), precision=inv(PRECISION, v.precision),
                tile_e=v.tile_e, elems_per_thread=v.elems_per_thread, split_i=v.split_i, unroll=v.unroll,
                prefetch_smem=v.prefetch_smem, tail_free=v.tail_free, stages=v.stages, ctas_per_sm=v.ctas_per_sm,
                out_buffers=v.out_buffers, store_rows=v.store_rows, max_ctas=v.max_ctas, mma_order=v.mma_order,
                a_operand=v.a_operand)


def variant_default(kernel: Kernel, E: int, N: int, F: int, layout="elem", precision="fp32") -> lc_variant:
    v = lc_variant()
    check(load().lc_variant_default(kernel.handle, E, N, F, LAYOUT[layout], PRECISION[precision],
                                    ctypes.byref(v)), "lc_variant_default")
    return v


def variant_validate(kernel: Kernel, E: int, N: int, F: int, v: lc_variant) -> int:
    return load().lc_variant_validate(kernel.handle, E, N, F, ctypes.byref(v))


def variant_plan(kernel: Kernel, E: int, N: int, F: int, v: lc_variant) -> dict:
    """The launch plan (lc_variant_plan) of a valid descriptor, as a dict."""
    p = lc_plan()
    p.struct_size = ctypes.sizeof(lc_plan)
    check(load().lc_variant_plan(kernel.handle, E, N, F, ctypes.byref(v), ctypes.byref(p)), "lc_variant_plan")
    return {n: getattr(p, n) for n, _ in lc_plan._fields_ if n != "struct_size"}


def lc_contract(kernel: Kernel, v: lc_variant, D_ptr: int, u_ptr: int, out_ptr: int, E: int, N: int, F: int,
                stream_ptr: int) -> int:
    return load().lc_contract(kernel.handle, ctypes.byref(v), D_ptr, u_ptr, out_ptr, E, N, F, stream_ptr)


def contract(kernel: Kernel, v: lc_variant, D, u, out=None, stream=None):
    """Enqueue the contraction on torch CUDA tensors. Returns ``out``.

    D: (F, N, N). u: (E, N) element-major or (N, E) node-major (per v.layout).
    out: (F, E, N) or (F, N, E); allocated with torch if not given.
    """
    import torch
    F, N, _ = D.shape
    node = v.layout == LAYOUT["node"]
    E = u.shape[1] if node else u.shape[0]
    if out is None:
        out = torch.empty((F, N, E) if node else (F, E, N), dtype=u.dtype, device=u.device)
    for t in (D, u, out):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("D, u and out must be contiguous CUDA tensors")
    st = lc_contract(kernel, v, D.data_ptr(), u.data_ptr(), out.data_ptr(), E, N, F, _stream_ptr(stream))
    check(st, "lc_contract")
    return out


GEO_DOMAIN = "{ [d,f,e,i,j]: 0<=d<F and 0<=f<F and 0<=e<E and 0<=i,j<N }"
GEO_INSTRUCTION = "out[d,e,i] = sum((f,j), G[e,d,f]*D[f,i,j]*u[e,j])"


def contract_geo(kernel: Kernel, v: lc_variant, D, u, r, out=None, stream=None):
    """Volume derivative with per-element geometric factors (lc_contract_geo) on torch CUDA
    tensors: D (F, N, N), u (E, N) or (N, E), r (E, F, F) element-major or (F, F, E)
    node-major; returns out (F, E, N) or (F, N, E)."""
    import torch
    F, N, _ = D.shape
    node = v.layout == LAYOUT["node"]
    E = u.shape[1] if node else u.shape[0]
    if out is None:
        out = torch.empty((F, N, E) if node else (F, E, N), dtype=u.dtype, device=u.device)
    for t in (D, u, r, out):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("D, u, r and out must be contiguous CUDA tensors")
    check(load().lc_contract_geo(kernel.handle, ctypes.byref(v), D.data_ptr(), u.data_ptr(), r.data_ptr(),
                                 out.data_ptr(), E, N, F, _stream_ptr(stream)), "lc_contract_geo")
    return out


LIFT_DOMAIN = "{ [e,i,f,p]: 0<=e<E and 0<=i<N and 0<=f<Nf and 0<=p<Nfp }"
LIFT_INSTRUCTION = "out[e,i] = sum((f,p), L[i,f,p]*s[e,f]*(u[e,fmask[f,p]] - u[vmapP[e,f,p]]))"


def lift(kernel: Kernel, v: lc_variant, L, fmask, vmapP, s, u, out=None, accumulate=False, stream=None):
    """Surface lift of the dG operator (lc_lift) on torch CUDA tensors: L (N, Nf*Nfp) float,
    fmask (Nf*Nfp,) int32, vmapP (E, Nf*Nfp) int32, s (E, Nf) float, u (E, N) float; returns
    out (E, N) (added to when accumulate)."""
    import torch
    E, N = u.shape
    Nf = s.shape[1]
    M = L.shape[1]
    if out is None:
        out = torch.zeros((E, N), dtype=torch.float32, device=u.device)
    for t in (L, fmask, vmapP, s, u, out):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("every array must be a contiguous CUDA tensor")
    check(load().lc_lift(kernel.handle, ctypes.byref(v), L.data_ptr(), fmask.data_ptr(), vmapP.data_ptr(),
                         s.data_ptr(), u.data_ptr(), out.data_ptr(), E, N, Nf, M // Nf, 1 if accumulate else 0,
                         _stream_ptr(stream)), "lc_lift")
    return out


def contract_host(kernel: Kernel, v: lc_variant, D_host, u_host, out_host, D_dev, u_dev, out_dev, stream=None):
    """Host arrays in, host array out, through the caller's device buffers (lc_contract_host)."""
    F, N, _ = D_host.shape
    node = v.layout == LAYOUT["node"]
    E = u_host.shape[1] if node else u_host.shape[0]
    st = load().lc_contract_host(kernel.handle, ctypes.byref(v), D_host.data_ptr(), u_host.data_ptr(),
                                 out_host.data_ptr(), E, N, F, D_dev.data_ptr(), u_dev.data_ptr(),
                                 out_dev.data_ptr(), _stream_ptr(stream))
    check(st, "lc_contract_host")
    return out_host


def device_error(clear: bool = True) -> int:
    return load().lc_device_error(1 if clear else 0)


def error_norm(out, ref, stream=None):
    """Relative Frobenius error ||out - ref|| / ||ref|| computed in FP64 on the GPU."""
    import torch
    lib = load()
    n = out.numel()
    assert ref.numel() == n and ref.dtype == torch.float64
    ws = ctypes.c_size_t(0)
    check(lib.lc_error_norm_workspace_size(n, ctypes.byref(ws)), "lc_error_norm_workspace_size")
    work = torch.empty(ws.value // 8 + 2, dtype=torch.float64, device=out.device)
    sums = torch.empty(2, dtype=torch.float64, device=out.device)
    dt = DTYPE_F64 if out.dtype == torch.float64 else DTYPE_F32
    check(lib.lc_error_norm(out.data_ptr(), dt, ref.data_ptr(), n, sums.data_ptr(), work.data_ptr(), ws.value,
                            _stream_ptr(stream)), "lc_error_norm")
    s = sums.cpu().tolist()
    return (s[0] / s[1]) ** 0.5 if s[1] > 0 else s[0] ** 0.5


def device_info():
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(load().lc_device_info(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "lc_device_info")
    return dict(sm_count=a.value, cc=(b.value, c.value))


class GroupedPlan:
    """One persistent launch over several problems (lc_grouped_plan_create), optionally a CUDA graph.

    groups: list of (D, u, out) torch CUDA tensors (out per the variant's layout). The plan keeps
    references to the tensors and to its workspace, which must stay alive while it is used.
    """

    def __init__(self, kernel: Kernel, v: lc_variant, groups, use_graph: bool = True, stream=None):
        import torch
        lib = load()
        node = v.layout == LAYOUT["node"]
        arr = (lc_group * len(groups))()
        for k, (D, u, out) in enumerate(groups):
            F, N, _ = D.shape
            arr[k].E = u.shape[1] if node else u.shape[0]
            arr[k].N, arr[k].F = N, F
            arr[k].D_dev, arr[k].u_dev, arr[k].out_dev = D.data_ptr(), u.data_ptr(), out.data_ptr()
        need = ctypes.c_size_t(0)
        check(lib.lc_grouped_workspace_size(kernel.handle, ctypes.byref(v), arr, len(groups), ctypes.byref(need)),
              "lc_grouped_workspace_size")
        dev = groups[0][0].device
        self.workspace = torch.empty(max(16, need.value), dtype=torch.uint8, device=dev)
        self._keep = (groups, kernel, v)
        h = ctypes.c_void_p()
        check(lib.lc_grouped_plan_create(kernel.handle, ctypes.byref(v), arr, len(groups), self.workspace.data_ptr(),
                                         need.value, 1 if use_graph else 0, _stream_ptr(stream), ctypes.byref(h)),
              "lc_grouped_plan_create")
        self._h = h
        self._lib = lib

    def run(self, stream=None):
        check(self._lib.lc_grouped_run(self._h, _stream_ptr(stream)), "lc_grouped_run")

    def info(self):
        g, sgs = ctypes.c_int32(), ctypes.c_int32()
        check(self._lib.lc_grouped_plan_info(self._h, ctypes.byref(g), ctypes.byref(sgs)), "lc_grouped_plan_info")
        return dict(grid=g.value, segments=sgs.value)

    def group_variant(self, k: int) -> lc_variant:
        """The descriptor that serves group k (lc_grouped_plan_group)."""
        v = lc_variant()
        check(self._lib.lc_grouped_plan_group(self._h, k, ctypes.byref(v)), "lc_grouped_plan_group")
        return v

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lc_grouped_plan_destroy(self._h)
            self._h = None


def enumerate_variants(kernel: Kernel, E: int, N: int, F: int, layout="elem", precision="fp32"):
    """The autotuner's candidate descriptors for a problem (valid ones, fixed order)."""
    lib = load()
    cap = 256
    arr = (lc_variant * cap)()
    n = ctypes.c_int32(0)
    check(lib.lc_enumerate_variants(kernel.handle, E, N, F, LAYOUT[layout], PRECISION[precision], arr, cap,
                                    ctypes.byref(n)), "lc_enumerate_variants")
    return [arr[q] for q in range(n.value)]


def autotune(kernel: Kernel, D, u, out, layout="elem", precision="fp32", reps=3, stream=None):
    """Time every candidate on (D, u, out); returns [(ms, lc_variant)] fastest first."""
    lib = load()
    F, N, _ = D.shape
    E = u.shape[1] if layout == "node" else u.shape[0]
    cap = 256
    arr = (lc_variant * cap)()
    ms = (ctypes.c_float * cap)()
    n = ctypes.c_int32(0)
    check(lib.lc_autotune(kernel.handle, E, N, F, LAYOUT[layout], PRECISION[precision], D.data_ptr(), u.data_ptr(),
                          out.data_ptr(), reps, arr, ms, cap, ctypes.byref(n), _stream_ptr(stream)), "lc_autotune")
    return [(float(ms[q]), arr[q]) for q in range(n.value)]


def mlp_param_count(din: int) -> int:
    n = ctypes.c_int64(0)
    check(load().lc_mlp_param_count(din, ctypes.byref(n)), "lc_mlp_param_count")
    return n.value


def mlp_forward(params, X, stream=None):
    """Predictions for the rows of X (float32 CUDA tensors)."""
    import torch
    n, din = X.shape
    y = torch.empty(n, dtype=torch.float32, device=X.device)
    check(load().lc_mlp_forward(params.data_ptr(), X.data_ptr(), n, din, y.data_ptr(), _stream_ptr(stream)),
          "lc_mlp_forward")
    return y


def mlp_loss_grad(params, X, t, workspace=None, stream=None):
    """(loss, grad) of the mean squared error, computed by the library's kernels."""
    import torch
    lib = load()
    n, din = X.shape
    ws = ctypes.c_size_t(0)
    check(lib.lc_mlp_workspace_size(din, ctypes.byref(ws)), "lc_mlp_workspace_size")
    if workspace is None or workspace.numel() * workspace.element_size() < ws.value:
        workspace = torch.empty(ws.value // 4 + 4, dtype=torch.float32, device=X.device)
    out = torch.empty(params.numel() + 1, dtype=torch.float32, device=X.device)
    check(lib.lc_mlp_loss_grad(params.data_ptr(), X.data_ptr(), t.data_ptr(), n, din, out.data_ptr(),
                               workspace.data_ptr(), ws.value, _stream_ptr(stream)), "lc_mlp_loss_grad")
    return out[-1], out[:-1]


def mlp_adam_step(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(load().lc_mlp_adam_step(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), params.numel(),
                                  step, lr, beta1, beta2, eps, _stream_ptr(stream)), "lc_mlp_adam_step")


def variant_features(kernel: Kernel, E: int, N: int, F: int, layout, precision, v: lc_variant):
    """The cost model's LC_FEATURES inputs for descriptor v on a problem (lc_variant_features)."""
    import numpy as np
    x = np.zeros(FEATURES, dtype=np.float32)
    check(load().lc_variant_features(kernel.handle, E, N, F, LAYOUT[layout] if isinstance(layout, str) else layout,
                                     PRECISION[precision] if isinstance(precision, str) else precision,
                                     ctypes.byref(v), x.ctypes.data_as(ctypes.c_void_p)), "lc_variant_features")
    return x


def pick_variant(kernel: Kernel, E: int, N: int, F: int, layout, precision, params, workspace=None, stream=None):
    """(descriptor, predicted log ms) picked by the trained network `params` (lc_pick_variant),
    or by an ensemble when `params` is 2-D, one network's parameters per row
    (lc_pick_variant_ensemble)."""
    import torch
    lib = load()
    need = ctypes.c_size_t(0)
    check(lib.lc_pick_workspace_size(ctypes.byref(need)), "lc_pick_workspace_size")
    if workspace is None or workspace.numel() * workspace.element_size() < need.value:
        workspace = torch.empty(need.value // 4 + 4, dtype=torch.float32, device=params.device)
    v = lc_variant()
    pred = ctypes.c_float(0.0)
    if params.dim() == 2:
        params = params.contiguous()
        check(lib.lc_pick_variant_ensemble(kernel.handle, E, N, F, LAYOUT[layout], PRECISION[precision],
                                           params.data_ptr(), params.shape[0], workspace.data_ptr(), need.value,
                                           ctypes.byref(v), ctypes.byref(pred), _stream_ptr(stream)),
              "lc_pick_variant_ensemble")
    else:
        check(lib.lc_pick_variant(kernel.handle, E, N, F, LAYOUT[layout], PRECISION[precision], params.data_ptr(),
                                  workspace.data_ptr(), need.value, ctypes.byref(v), ctypes.byref(pred),
                                  _stream_ptr(stream)), "lc_pick_variant")
    return v, pred.value


def kernel_args(kernel: Kernel) -> dict:
    """Argument names in call order: {"arrays": [...], "params": [...], "dims": [...]}."""
    lib = load()
    na, npar, nd = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(lib.lc_kernel_signature(kernel.handle, ctypes.byref(na), ctypes.byref(npar), ctypes.byref(nd)),
          "lc_kernel_signature")
    buf = ctypes.create_string_buffer(256)

    def names(what, n):
        out = []
        for q in range(n):
            check(lib.lc_kernel_arg_name(kernel.handle, what, q, buf, 256), "lc_kernel_arg_name")
            out.append(buf.value.decode())
        return out
    return dict(arrays=names(0, na.value), params=names(1, npar.value), dims=names(2, nd.value))


def elementwise_source(kernel: Kernel, v: lc_variant, extents) -> str:
    """The CUDA source lc_elementwise compiles for this descriptor and these extents."""
    lib = load()
    ext = (ctypes.c_int64 * 2)(*(list(extents) + [1])[:2])
    need = ctypes.c_size_t(0)
    lib.lc_elementwise_source(kernel.handle, ctypes.byref(v), ext, None, 0, ctypes.byref(need))
    buf = ctypes.create_string_buffer(need.value)
    check(lib.lc_elementwise_source(kernel.handle, ctypes.byref(v), ext, buf, need.value, ctypes.byref(need)),
          "lc_elementwise_source")
    return buf.value.decode()


def elementwise(kernel: Kernel, v: lc_variant, arrays, params=(), extents=None, stream=None):
    """Run an elementwise kernel (lc_elementwise). arrays: torch CUDA float32 tensors in
    signature order (arrays[0] is the output); params: scalars in order; extents: one per
    iname (default: the output's shape). Returns arrays[0]."""
    lib = load()
    ext = list(extents) if extents is not None else list(arrays[0].shape)
    e_arr = (ctypes.c_int64 * max(1, len(ext)))(*ext)
    ptrs = (ctypes.c_void_p * len(arrays))(*[a.data_ptr() for a in arrays])
    par = (ctypes.c_double * max(1, len(params)))(*params)
    check(lib.lc_elementwise(kernel.handle, ctypes.byref(v), e_arr, ptrs, par, _stream_ptr(stream)),
          "lc_elementwise")
    return arrays[0]
