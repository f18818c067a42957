"""ctypes binding of libdualk.so (include/dualk.h), names matching the C ABI.

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. Tensors are torch CUDA tensors (PyTorch provides device memory and streams);
outputs are allocated here with torch when the caller does not pass them. If the
library is not built, or no sm_10x device is visible, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdualk.so")

DK_OK = 0
DK_C64, DK_C128, DK_SPLIT_BF16 = 0, 1, 2
DK_PREC_F32, DK_PREC_F64, DK_PREC_BF16X3 = 0, 1, 2
DK_BLOCK_TCGEN05, DK_BLOCK_MMA_SYNC = 0, 1

_STATUS_NAMES = {0: "DK_OK", 1: "DK_ERR_ARG", 2: "DK_ERR_UNSUPPORTED", 3: "DK_ERR_CUDA",
                 4: "DK_ERR_TIMEOUT", 5: "DK_ERR_WORKSPACE", 6: "DK_ERR_NO_DEVICE"}

EXPORTED = ("dk_create", "dk_destroy", "dk_error_string", "dk_sync_status", "dk_mps_bytes",
            "dk_mps_build", "dk_gram_tile", "dk_dual_kernel_rows", "dk_gram_config_count",
            "dk_gram_config_info", "dk_set_gram_config", "dk_selftest_wait_timeout", "dk_self_overlap",
            "dk_svm_ovo_train", "dk_svm_ovo_predict", "dk_gram_stats", "dk_pca_workspace_bytes", "dk_pca_fit",
            "dk_pca_transform", "dk_pca_fit_noalloc", "dk_mps_build_blocks", "dk_block_states_bytes",
            "dk_block_states", "dk_gram_blocks", "dk_gram_sweep", "dk_workspace_bytes",
            "dk_set_block_gram_form", "dk_block_states_workspace_bytes", "dk_gram_blocks_workspace_bytes",
            "dk_gram_refine", "dk_gram_refine_workspace_bytes", "dk_gram_blocks_refine", "dk_mps_split32")
# Entries with K_q above this are recomputed after every FP32 / split-BF16 Gram, rows and
# block-Gram call of the binding (dk_gram_refine, dk_gram_blocks_refine; refine=None: not).
REFINE_TAU = 0.02  # DK_REFINE_TAU
SVM_MAX_SAMPLES = 4096  # DK_SVM_MAX_SAMPLES
PCA_MAX_FEATURES = 4096  # DK_PCA_MAX_FEATURES
PCA_NOALLOC_MAX_FEATURES = 256  # DK_PCA_NOALLOC_MAX_FEATURES


class DualKError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_STATUS_NAMES.get(status, status)} ({_lib().dk_error_string(status).decode()})")


class _Fmap(ctypes.Structure):
    _fields_ = [("reps", ctypes.c_int), ("angle_scale", ctypes.c_float),
                ("entangle", ctypes.c_int), ("chi_max", ctypes.c_int), ("qr_prec", ctypes.c_int),
                ("block", ctypes.c_int)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2602_01330_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    lib.dk_create.argtypes = [ctypes.POINTER(vp), i32]
    lib.dk_create.restype = i32
    lib.dk_destroy.argtypes = [vp]
    lib.dk_destroy.restype = None
    lib.dk_error_string.argtypes = [i32]
    lib.dk_error_string.restype = ctypes.c_char_p
    lib.dk_sync_status.argtypes = [vp, vp]
    lib.dk_sync_status.restype = i32
    lib.dk_mps_bytes.argtypes = [i32, i32, i32, i32]
    lib.dk_mps_bytes.restype = ctypes.c_size_t
    lib.dk_mps_build.argtypes = [vp, vp, i32, i32, ctypes.POINTER(_Fmap), i32, vp, vp, vp, vp]
    lib.dk_mps_build.restype = i32
    lib.dk_mps_build_blocks.argtypes = [vp, vp, i32, i32, ctypes.POINTER(_Fmap), i32, ctypes.c_double, i32, vp, vp,
                                        vp, vp, vp]
    lib.dk_mps_build_blocks.restype = i32
    lib.dk_workspace_bytes.argtypes = [i32, i32, i32, i32]
    lib.dk_workspace_bytes.restype = ctypes.c_size_t
    lib.dk_gram_sweep.argtypes = [vp, ctypes.POINTER(_SweepItem), i32, i32, i32, i32, f32, i32, vp, ctypes.c_size_t,
                                  vp]
    lib.dk_gram_sweep.restype = i32
    lib.dk_block_states_bytes.argtypes = [i32, i32, i32]
    lib.dk_block_states_bytes.restype = ctypes.c_size_t
    sz = ctypes.c_size_t
    lib.dk_block_states.argtypes = [vp, vp, i32, i32, ctypes.POINTER(_Fmap), i32, i32, vp, vp, vp, sz, vp]
    lib.dk_block_states.restype = i32
    lib.dk_block_states_workspace_bytes.argtypes = [vp, i32, i32, i32, i32]
    lib.dk_block_states_workspace_bytes.restype = sz
    lib.dk_gram_blocks.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, i32, vp, vp, vp, vp, f32, f32,
                                   i32, vp, vp, vp, vp, i64, i32, vp, sz, vp]
    lib.dk_gram_blocks.restype = i32
    lib.dk_gram_blocks_workspace_bytes.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32]
    lib.dk_gram_blocks_workspace_bytes.restype = sz
    lib.dk_gram_tile.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, i32, i32,
                                 vp, vp, vp, vp, f32, f32, i32, vp, vp, vp, vp, i64, i32, vp]
    lib.dk_gram_tile.restype = i32
    lib.dk_dual_kernel_rows.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, i32, i32, i32, i32,
                                        f32, f32, i32, vp, vp, vp, vp, vp]
    lib.dk_dual_kernel_rows.restype = i32
    lib.dk_gram_refine.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp, f32, f32, f32,
                                   vp, vp, vp, vp, i64, i32, vp, ctypes.c_size_t, vp]
    lib.dk_gram_refine.restype = i32
    lib.dk_gram_blocks_refine.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp, f32, f32,
                                          f32, vp, vp, vp, vp, i64, i32, vp]
    lib.dk_gram_blocks_refine.restype = i32
    lib.dk_mps_split32.argtypes = [vp, vp, i32, i32, vp, ctypes.c_size_t, vp]
    lib.dk_mps_split32.restype = i32
    lib.dk_gram_refine_workspace_bytes.argtypes = [i32, i32]
    lib.dk_gram_refine_workspace_bytes.restype = ctypes.c_size_t
    lib.dk_gram_config_count.argtypes = [i32, i32]
    lib.dk_gram_config_count.restype = i32
    ip = ctypes.POINTER(ctypes.c_int)
    lib.dk_gram_config_info.argtypes = [i32, i32, i32, ip, ip, ip]
    lib.dk_gram_config_info.restype = i32
    lib.dk_set_gram_config.argtypes = [vp, i32]
    lib.dk_set_gram_config.restype = i32
    lib.dk_set_block_gram_form.argtypes = [vp, i32]
    lib.dk_set_block_gram_form.restype = i32
    lib.dk_self_overlap.argtypes = [vp, vp, i32, i32, i32, i32, i32, vp, vp]
    lib.dk_self_overlap.restype = i32
    lib.dk_selftest_wait_timeout.argtypes = [vp, ctypes.c_ulonglong, vp]
    lib.dk_selftest_wait_timeout.restype = i32
    lib.dk_pca_workspace_bytes.argtypes = [i32]
    lib.dk_pca_workspace_bytes.restype = ctypes.c_size_t
    lib.dk_pca_fit.argtypes = [vp, vp, i32, i32, i32, i32, vp, ctypes.c_size_t, vp, vp, vp, vp, vp, vp]
    lib.dk_pca_fit.restype = i32
    lib.dk_pca_fit_noalloc.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.dk_pca_fit_noalloc.restype = i32
    lib.dk_pca_transform.argtypes = [vp, vp, i32, i32, vp, vp, vp, i32, i32, f32, vp, vp, vp, vp]
    lib.dk_pca_transform.restype = i32
    lib.dk_gram_stats.argtypes = [vp, vp, vp, i64, i32, i32, i32, vp, vp]
    lib.dk_gram_stats.restype = i32
    lib.dk_svm_ovo_train.argtypes = [vp, vp, vp, i64, i32, i32, vp, vp, vp, vp, i32, vp, i32, f32, i32, vp, vp, vp,
                                     vp]
    lib.dk_svm_ovo_train.restype = i32
    lib.dk_svm_ovo_predict.argtypes = [vp, vp, vp, i64, i32, i32, i32, vp, vp, vp, i32, vp, vp, i32, vp, vp, i32, vp,
                                       vp, vp]
    lib.dk_svm_ovo_predict.restype = i32
    _LIB = lib
    return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(status: int, what: str):
    if status != DK_OK:
        raise DualKError(status, what)


def _need_cuda(t, name, dtype=None):
    if t is None:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")


@dataclass
class FeatureMap:
    """ZZ-chain feature map: reps x (H, RZ(angle_scale x_i), RZZ chain); see include/dualk.h.
    block = b >= 1 keeps only the RZZ inside blocks of b consecutive qubits (block product form)."""
    reps: int = 2
    angle_scale: float = 2.0
    entangle: bool = True
    chi_max: int = 4
    qr_prec: int = 0  # DK_PREC_F32 / DK_PREC_F64: QR arithmetic of complex64 bond-4 builds
    block: int = 0

    def _c(self):
        return _Fmap(self.reps, self.angle_scale, 1 if self.entangle else 0, self.chi_max, self.qr_prec,
                     self.block)


@dataclass
class MPS:
    """Device MPS batch as written by mps_build (site-major, see include/dualk.h)."""
    data: torch.Tensor        # uint8 bytes
    m: int
    n: int
    chi_max: int
    dtype: int                # DK_C64 / DK_C128
    bond_dims: torch.Tensor   # int32, n + 1
    log_norm: torch.Tensor    # float32, m
    x: torch.Tensor           # float32 m x n features it was built from
    norms: dict | None = None  # precision -> log_norm computed with that arithmetic
    fmap: "FeatureMap | None" = None  # the feature map it was built with
    split: torch.Tensor | None = None  # dk_mps_split32 operands (bond 32), made on first use

    def log_norm_for(self, ctx: "Context", prec: int, stream=None) -> torch.Tensor:
        """ln-norms matching the Gram precision `prec` (dk_self_overlap when not built in)."""
        native = DK_PREC_F32 if self.dtype == DK_C64 else DK_PREC_F64
        if prec == native:
            return self.log_norm
        if self.norms is None:
            self.norms = {}
        if prec not in self.norms:
            self.norms[prec] = self_overlap(ctx, self, prec, stream=stream)
        return self.norms[prec]

    def split_for(self, ctx: "Context", stream=None) -> torch.Tensor:
        """The split-BF16 operands of this bond-32 complex64 MPS (dk_mps_split32), which the
        BF16X3 Gram calls read instead of the site tensors; made once and kept."""
        if self.chi_max != 32 or self.dtype != DK_C64:
            raise ValueError("split operands exist for bond-32 complex64 MPS only")
        if self.split is None:
            nbytes = int(_lib().dk_mps_bytes(self.m, self.n, 32, DK_SPLIT_BF16))
            split = torch.empty(nbytes, dtype=torch.uint8, device=self.data.device)
            _check(_lib().dk_mps_split32(ctx.handle, _ptr(self.data), self.m, self.n, _ptr(split), nbytes,
                                         _stream(stream)), "dk_mps_split32")
            self.split = split
        return self.split

    def complex_view(self):
        """[site][sample][s][j][l] view of the compact block layout (see include/dualk.h)."""
        ct = torch.complex64 if self.dtype == DK_C64 else torch.complex128
        return self.data.view(ct).view(self.n, self.m, 2, self.chi_max // 2, self.chi_max)


class Context:
    """dk_ctx on one device."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(_lib().dk_create(ctypes.byref(h), int(device)), "dk_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            _lib().dk_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass

    def sync_status(self, stream=None):
        _check(_lib().dk_sync_status(self.handle, _stream(stream)), "dk_sync_status")

    def selftest_wait_timeout(self, limit_ns: int = 50_000_000, stream=None):
        """dk_selftest_wait_timeout: a bounded wait that must time out (see include/dualk.h)."""
        _check(_lib().dk_selftest_wait_timeout(self.handle, int(limit_ns), _stream(stream)),
               "dk_selftest_wait_timeout")

    def set_gram_config(self, cfg_id: int):
        """dk_set_gram_config: 0 = built-in tile shape, 1..gram_config_count() = a fixed one."""
        _check(_lib().dk_set_gram_config(self.handle, int(cfg_id)), "dk_set_gram_config")

    def set_block_gram_form(self, form: int):
        """dk_set_block_gram_form: DK_BLOCK_TCGEN05 (default) or DK_BLOCK_MMA_SYNC kernels for
        the split-BF16 block states' self-norms and Gram; build states and Gram in one form."""
        _check(_lib().dk_set_block_gram_form(self.handle, int(form)), "dk_set_block_gram_form")


def gram_config_count(dtype: int = DK_C64, chi_max: int = 4) -> int:
    return int(_lib().dk_gram_config_count(dtype, chi_max))


def gram_config_info(cfg_id: int, dtype: int = DK_C64, chi_max: int = 4):
    """(tile_rows, tile_cols, threads) of a Gram tile shape."""
    r, c, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib().dk_gram_config_info(dtype, chi_max, cfg_id, ctypes.byref(r), ctypes.byref(c), ctypes.byref(t)),
           "dk_gram_config_info")
    return r.value, c.value, t.value


def mps_bytes(m: int, n: int, chi_max: int, dtype: int = DK_C64) -> int:
    return int(_lib().dk_mps_bytes(m, n, chi_max, dtype))


def mps_build(ctx: Context, x: torch.Tensor, fmap: FeatureMap, dtype: int = DK_C64,
              out: torch.Tensor | None = None, stream=None, bond: torch.Tensor | None = None,
              log_norm: torch.Tensor | None = None) -> MPS:
    """dk_mps_build: MPS of |psi(x_i)> for the rows of x (m x n float32, CUDA).

    out / bond / log_norm may be preallocated (bytes, n + 1 int32, m float32)."""
    _need_cuda(x, "x", torch.float32)
    m, n = x.shape
    nbytes = mps_bytes(m, n, fmap.chi_max, dtype)
    if out is None:
        out = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    elif out.numel() * out.element_size() < nbytes:
        raise ValueError("out is too small for the MPS")
    if bond is None:
        bond = torch.empty(n + 1, dtype=torch.int32, device=x.device)
    if log_norm is None:
        log_norm = torch.empty(m, dtype=torch.float32, device=x.device)
    _need_cuda(bond, "bond", torch.int32)
    _need_cuda(log_norm, "log_norm", torch.float32)
    lnorm = log_norm
    fm = fmap._c()
    _check(_lib().dk_mps_build(ctx.handle, _ptr(x), m, n, ctypes.byref(fm), dtype, _ptr(out), _ptr(bond),
                               _ptr(lnorm), _stream(stream)), "dk_mps_build")
    return MPS(out, m, n, fmap.chi_max, dtype, bond, lnorm, x, fmap=fmap)


class _SweepItem(ctypes.Structure):
    _fields_ = [("mps", ctypes.c_void_p), ("log_norm", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("k", ctypes.c_void_p), ("kq", ctypes.c_void_p), ("kc", ctypes.c_void_p), ("logkq", ctypes.c_void_p),
                ("ld", ctypes.c_longlong), ("m", ctypes.c_int), ("n", ctypes.c_int), ("tile_shape", ctypes.c_int)]


def gram_sweep(ctx: "Context", items, w: float = 0.5, prec: int | None = None, graph: bool = False, stream=None,
               ws: torch.Tensor | None = None):
    """dk_gram_sweep over items = [(MPS, out dict of m x m tensors, tile_shape id)], all with
    the same chi_max and dtype. graph=True records the launches once into a CUDA graph kept by
    the context and replays it on later calls with the same items (needs a non-default stream).
    ws: workspace of the refinement passes (refine_workspace(m, m) for the largest m), kept by
    the caller across calls (a recorded graph refers to it); None: per-entry norms."""
    first = items[0][0]
    prec = _default_prec(first) if prec is None else prec
    arr = (_SweepItem * len(items))()
    for t, (mps, out, tile) in enumerate(items):
        if mps.chi_max != first.chi_max or mps.dtype != first.dtype:
            raise ValueError("sweep items differ in chi_max or dtype")
        ln = mps.log_norm_for(ctx, prec, stream)
        arr[t] = _SweepItem(_ptr(mps.data), _ptr(ln), _ptr(mps.x), _ptr(out.get("k")), _ptr(out.get("kq")),
                            _ptr(out.get("kc")), _ptr(out.get("logkq")), mps.m, mps.m, mps.n, int(tile))
    _check(_lib().dk_gram_sweep(ctx.handle, arr, len(items), first.chi_max, first.dtype, int(prec), float(w),
                                1 if graph else 0, _ptr(ws), 0 if ws is None else int(ws.numel()), _stream(stream)),
           "dk_gram_sweep")


DK_ENT_CHAIN, DK_ENT_FULL = 0, 1


def mps_build_blocks(ctx: Context, x: torch.Tensor, fmap: FeatureMap, entangler: int = DK_ENT_FULL,
                     cutoff: float = 1e-10, dtype: int = DK_C64, stream=None):
    """dk_mps_build_blocks: MPS of a block-structured map (fmap.block qubits per block) from
    block statevectors with SVD truncation. Returns (MPS, discarded weight per sample)."""
    _need_cuda(x, "x", torch.float32)
    m, n = x.shape
    out = torch.empty(mps_bytes(m, n, fmap.chi_max, dtype), dtype=torch.uint8, device=x.device)
    bond = torch.empty(n + 1, dtype=torch.int32, device=x.device)
    log_norm = torch.empty(m, dtype=torch.float32, device=x.device)
    disc = torch.empty(m, dtype=torch.float32, device=x.device)
    fm = fmap._c()
    _check(_lib().dk_mps_build_blocks(ctx.handle, _ptr(x), m, n, ctypes.byref(fm), int(entangler), float(cutoff),
                                      dtype, _ptr(out), _ptr(bond), _ptr(log_norm), _ptr(disc), _stream(stream)),
           "dk_mps_build_blocks")
    return MPS(out, m, n, fmap.chi_max, dtype, bond, log_norm, x, fmap=fmap), disc


@dataclass
class BlockStates:
    """Block statevectors written by dk_block_states ([block][sample][dpad] complex64)."""
    data: torch.Tensor      # uint8 bytes
    m: int
    n: int
    block: int
    log_norm: torch.Tensor  # float32, m
    x: torch.Tensor         # float32 m x n features
    prec: int = 0           # DK_PREC_F32 (complex64) or DK_PREC_BF16X3 (split-BF16 chunk rows)


def block_states(ctx: Context, x: torch.Tensor, fmap: FeatureMap, entangler: int = DK_ENT_FULL,
                 prec: int = DK_PREC_F32, stream=None) -> BlockStates:
    """dk_block_states: per-block statevectors of a block-structured map (fmap.block qubits),
    laid out for the Gram precision `prec` (F32 CUDA cores or BF16X3 tensor cores)."""
    _need_cuda(x, "x", torch.float32)
    m, n = x.shape
    nbytes = int(_lib().dk_block_states_bytes(m, n, int(fmap.block)))
    if nbytes == 0:
        raise ValueError(f"block {fmap.block} is outside the supported range for n = {n}")
    out = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    log_norm = torch.empty(m, dtype=torch.float32, device=x.device)
    ws_bytes = int(_lib().dk_block_states_workspace_bytes(ctx.handle, m, n, int(fmap.block), int(prec)))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=x.device) if ws_bytes else None
    fm = fmap._c()
    _check(_lib().dk_block_states(ctx.handle, _ptr(x), m, n, ctypes.byref(fm), int(entangler), int(prec), _ptr(out),
                                  _ptr(log_norm), _ptr(ws), ws_bytes, _stream(stream)), "dk_block_states")
    return BlockStates(out, m, n, fmap.block, log_norm, x, int(prec))


def gram_blocks(ctx: Context, rows: BlockStates, cols: BlockStates | None = None, gamma: float | None = None,
                w: float = 0.5, want=("k", "kq", "kc", "logkq"), stream=None,
                refine: float | None = REFINE_TAU) -> dict:
    """dk_gram_blocks: K, K_q, K_c, log K_q of rows x cols (symmetric when cols is None), then
    dk_gram_blocks_refine with tau = refine (None: no refinement)."""
    symmetric = cols is None
    cols = rows if cols is None else cols
    if rows.n != cols.n or rows.block != cols.block or rows.prec != cols.prec:
        raise ValueError("row and column states differ in n, block or precision")
    gamma = 1.0 / rows.n if gamma is None else gamma
    out = _outs((rows.m, cols.m), rows.data.device, want)
    with_kc = out.get("kc") is not None or (out.get("k") is not None and w != 1.0)
    ws_bytes = int(_lib().dk_gram_blocks_workspace_bytes(ctx.handle, rows.n, rows.block, rows.m, cols.m, rows.prec,
                                                         1 if symmetric else 0, 1 if with_kc else 0))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=rows.data.device) if ws_bytes else None
    _check(_lib().dk_gram_blocks(ctx.handle, _ptr(rows.data), rows.m, _ptr(cols.data), cols.m, rows.n, rows.block,
                                 0, rows.m, 0, cols.m, _ptr(rows.log_norm), _ptr(cols.log_norm), _ptr(rows.x),
                                 _ptr(cols.x), float(gamma), float(w), rows.prec, _ptr(out.get("k")),
                                 _ptr(out.get("kq")),
                                 _ptr(out.get("kc")), _ptr(out.get("logkq")), int(cols.m), 1 if symmetric else 0,
                                 _ptr(ws), ws_bytes, _stream(stream)), "dk_gram_blocks")
    if refine is not None and (out.get("kq") is not None or out.get("logkq") is not None):
        _check(_lib().dk_gram_blocks_refine(ctx.handle, _ptr(rows.data), rows.m, _ptr(cols.data), cols.m, rows.n,
                                            rows.block, rows.prec, 0, rows.m, 0, cols.m, _ptr(rows.x),
                                            _ptr(cols.x), float(gamma), float(w), float(refine),
                                            _ptr(out.get("k")), _ptr(out.get("kq")), _ptr(out.get("kc")),
                                            _ptr(out.get("logkq")), int(cols.m), 1 if symmetric else 0,
                                            _stream(stream)), "dk_gram_blocks_refine")
    return out


def self_overlap(ctx: Context, mps: "MPS", prec: int, out: torch.Tensor | None = None, stream=None):
    """dk_self_overlap: ln|<psi~|psi~>| per sample with the arithmetic of precision `prec`."""
    if out is None:
        out = torch.empty(mps.m, dtype=torch.float32, device=mps.data.device)
    _check(_lib().dk_self_overlap(ctx.handle, _ptr(mps.data), mps.m, mps.n, mps.chi_max, mps.dtype, int(prec),
                                  _ptr(out), _stream(stream)), "dk_self_overlap")
    return out


def _default_prec(mps):
    return DK_PREC_F32 if mps.dtype == DK_C64 else DK_PREC_F64


def _refinable(mps, prec):
    return mps.dtype == DK_C64 and mps.chi_max in (4, 8, 32) and prec in (DK_PREC_F32, DK_PREC_BF16X3)


def refine_workspace(rows_m: int, cols_m: int, device) -> torch.Tensor:
    """Scratch for dk_gram_refine's once-per-sample ln-norms (dk_gram_refine_workspace_bytes)."""
    return torch.empty(int(_lib().dk_gram_refine_workspace_bytes(int(rows_m), int(cols_m))), dtype=torch.uint8,
                       device=device)


def gram_refine(ctx: "Context", rows: "MPS", cols: "MPS", row0: int, nrows: int, col0: int, ncols: int, out: dict,
                ld: int, gamma: float, w: float, tau: float = REFINE_TAU, symmetric: bool = False, stream=None,
                ws: torch.Tensor | None = None):
    """dk_gram_refine: recompute the entries of a written block with K_q > tau in double-word
    FP32 (see include/dualk.h), with a workspace for once-per-sample ln-norms (allocated here
    when not given)."""
    if ws is None:
        ws = refine_workspace(rows.m, cols.m, rows.data.device)
    _check(_lib().dk_gram_refine(ctx.handle, _ptr(rows.data), rows.m, _ptr(cols.data), cols.m, rows.n,
                                 rows.chi_max, rows.dtype, row0, nrows, col0, ncols, _ptr(rows.x), _ptr(cols.x),
                                 float(gamma), float(w), float(tau), _ptr(out.get("k")), _ptr(out.get("kq")),
                                 _ptr(out.get("kc")), _ptr(out.get("logkq")), int(ld), 1 if symmetric else 0,
                                 _ptr(ws), int(ws.numel()), _stream(stream)), "dk_gram_refine")


def _outs(shape, device, want):
    return {k: (torch.empty(shape, dtype=torch.float32, device=device) if k in want else None)
            for k in ("k", "kq", "kc", "logkq")}


def _gram_operands(ctx: "Context", mps: MPS, prec: int, stream=None):
    """(buffer, dtype) a Gram call reads: the split operands for bond-32 split-BF16 Grams,
    the site tensors otherwise."""
    if prec == DK_PREC_BF16X3 and mps.chi_max == 32 and mps.dtype == DK_C64:
        return mps.split_for(ctx, stream), DK_SPLIT_BF16
    return mps.data, mps.dtype


def gram_tile(ctx: Context, rows: MPS, cols: MPS, row0: int = 0, nrows: int | None = None,
              col0: int = 0, ncols: int | None = None, gamma: float | None = None, w: float = 0.5,
              want=("k", "kq", "kc", "logkq"), symmetric: bool = False, out=None, ld: int | None = None,
              stream=None, prec: int | None = None, refine: float | None = REFINE_TAU,
              refine_ws: torch.Tensor | None = None):
    """dk_gram_tile: the (nrows x ncols) block of K, K_q, K_c, log K_q (dict of tensors),
    then dk_gram_refine with tau = refine for FP32 / split-BF16 blocks (None: no refinement;
    refine_ws: its workspace, allocated when not given)."""
    nrows = rows.m - row0 if nrows is None else nrows
    ncols = cols.m - col0 if ncols is None else ncols
    if rows.n != cols.n or rows.chi_max != cols.chi_max or rows.dtype != cols.dtype:
        raise ValueError("row and column MPS differ in n, chi_max or dtype")
    gamma = 1.0 / rows.n if gamma is None else gamma
    if out is None:
        out = _outs((nrows, ncols), rows.data.device, want)
        ld = ncols
    elif ld is None:
        raise ValueError("ld is required with caller-provided outputs")
    prec = _default_prec(rows) if prec is None else prec
    ln_r = rows.log_norm_for(ctx, prec, stream)
    ln_c = ln_r if cols is rows else cols.log_norm_for(ctx, prec, stream)
    buf_r, dt = _gram_operands(ctx, rows, prec, stream)
    buf_c = buf_r if cols is rows else _gram_operands(ctx, cols, prec, stream)[0]
    _check(_lib().dk_gram_tile(ctx.handle, _ptr(buf_r), rows.m, _ptr(buf_c), cols.m, rows.n,
                               rows.chi_max, dt, row0, nrows, col0, ncols, _ptr(ln_r),
                               _ptr(ln_c), _ptr(rows.x), _ptr(cols.x), float(gamma), float(w), prec,
                               _ptr(out.get("k")), _ptr(out.get("kq")), _ptr(out.get("kc")),
                               _ptr(out.get("logkq")), int(ld), 1 if symmetric else 0, _stream(stream)),
           "dk_gram_tile")
    if refine is not None and _refinable(rows, prec) and (out.get("kq") is not None or out.get("logkq") is not None):
        gram_refine(ctx, rows, cols, row0, nrows, col0, ncols, out, ld, gamma, w, refine, symmetric, stream,
                    ws=refine_ws)
    return out


def gram(ctx: Context, mps: MPS, gamma: float | None = None, w: float = 0.5,
         want=("k", "kq", "kc", "logkq"), stream=None, prec: int | None = None, refine: float | None = REFINE_TAU,
         refine_ws: torch.Tensor | None = None):
    """Full symmetric m x m Gram of one MPS batch (each unordered pair contracted once)."""
    return gram_tile(ctx, mps, mps, gamma=gamma, w=w, want=want, symmetric=True, stream=stream, prec=prec,
                     refine=refine, refine_ws=refine_ws)


def dual_kernel_rows(ctx: Context, test: MPS, train: MPS, gamma: float | None = None, w: float = 0.5,
                     want=("k", "kq", "kc", "logkq"), out=None, stream=None, prec: int | None = None,
                     refine: float | None = REFINE_TAU, refine_ws: torch.Tensor | None = None):
    """dk_dual_kernel_rows: the b x m block K(test, train), then dk_gram_refine (tau = refine)
    for FP32 / split-BF16 blocks."""
    if test.n != train.n or test.chi_max != train.chi_max or test.dtype != train.dtype:
        raise ValueError("test and train MPS differ in n, chi_max or dtype")
    gamma = 1.0 / train.n if gamma is None else gamma
    if out is None:
        out = _outs((test.m, train.m), train.data.device, want)
    prec = _default_prec(train) if prec is None else prec
    ln_te = test.log_norm_for(ctx, prec, stream)
    ln_tr = train.log_norm_for(ctx, prec, stream)
    buf_te, dt = _gram_operands(ctx, test, prec, stream)
    buf_tr = _gram_operands(ctx, train, prec, stream)[0]
    _check(_lib().dk_dual_kernel_rows(ctx.handle, _ptr(buf_te), _ptr(test.x), _ptr(ln_te), test.m,
                                      _ptr(buf_tr), _ptr(train.x), _ptr(ln_tr), train.m, train.n,
                                      train.chi_max, dt, float(gamma), float(w), prec,
                                      _ptr(out.get("k")), _ptr(out.get("kq")), _ptr(out.get("kc")),
                                      _ptr(out.get("logkq")), _stream(stream)),
           "dk_dual_kernel_rows")
    if refine is not None and _refinable(train, prec) and (out.get("kq") is not None or out.get("logkq") is not None):
        gram_refine(ctx, test, train, 0, test.m, 0, train.m, out, train.m, gamma, w, refine, False, stream,
                    ws=refine_ws)
    return out


def svm_ovo_train(ctx: Context, kq: torch.Tensor | None, kc: torch.Tensor | None, w: torch.Tensor,
                  C: torch.Tensor, idx: torch.Tensor, count: torch.Tensor, labels: torch.Tensor, n_class: int,
                  tol: float = 1e-3, max_iter: int = 1_000_000, out=None, stream=None):
    """dk_svm_ovo_train: one-against-one SVMs for n_jobs jobs (see include/dualk.h).

    kq / kc: kernel matrices (float32, row-major, same leading dimension); w, C: (n_jobs,)
    float32; idx: (n_jobs, m_max) int32; count: (n_jobs,) int32; labels: int32 per kernel row.
    Returns a dict with coef (n_jobs, P, m_max), bias (n_jobs, P) and iters (n_jobs, P)."""
    ref = kq if kq is not None else kc
    for t, name, dt in ((kq, "kq", torch.float32), (kc, "kc", torch.float32), (w, "w", torch.float32),
                        (C, "C", torch.float32), (idx, "idx", torch.int32), (count, "count", torch.int32),
                        (labels, "labels", torch.int32)):
        _need_cuda(t, name, dt)
    if kq is not None and kc is not None and kq.shape != kc.shape:
        raise ValueError("kq and kc differ in shape")
    n_jobs, m_max = idx.shape
    P = n_class * (n_class - 1) // 2
    if out is None:
        out = {"coef": torch.empty((n_jobs, P, m_max), dtype=torch.float32, device=ref.device),
               "bias": torch.empty((n_jobs, P), dtype=torch.float32, device=ref.device),
               "iters": torch.empty((n_jobs, P), dtype=torch.int32, device=ref.device)}
    if ref.dim() != 2 or ref.shape[0] != ref.shape[1]:
        raise ValueError("the training kernel must be a square matrix")
    _check(_lib().dk_svm_ovo_train(ctx.handle, _ptr(kq), _ptr(kc), int(ref.stride(0)), int(ref.shape[0]), n_jobs,
                                   _ptr(w), _ptr(C),
                                   _ptr(idx), _ptr(count), m_max, _ptr(labels), int(n_class), float(tol),
                                   int(max_iter), _ptr(out["coef"]), _ptr(out["bias"]), _ptr(out.get("iters")),
                                   _stream(stream)), "dk_svm_ovo_train")
    return out


def svm_ovo_predict(ctx: Context, kq: torch.Tensor | None, kc: torch.Tensor | None, w: torch.Tensor,
                    model: dict, n_class: int, rows: torch.Tensor | None = None,
                    row_count: torch.Tensor | None = None, r_max: int | None = None,
                    idx: torch.Tensor | None = None, count: torch.Tensor | None = None,
                    want_decision: bool = True, stream=None):
    """dk_svm_ovo_predict: decision values (n_jobs, r_max, P) and votes (n_jobs, r_max).

    rows (n_jobs, r_max) int32 or None (rows 0..r_max-1 of kq / kc); idx / count: the jobs'
    training lists as given to svm_ovo_train, or None for columns 0..m_max-1."""
    ref = kq if kq is not None else kc
    for t, name, dt in ((kq, "kq", torch.float32), (kc, "kc", torch.float32), (w, "w", torch.float32),
                        (rows, "rows", torch.int32), (row_count, "row_count", torch.int32),
                        (idx, "idx", torch.int32), (count, "count", torch.int32)):
        _need_cuda(t, name, dt)
    coef, bias = model["coef"], model["bias"]
    n_jobs, P, m_max = coef.shape
    if r_max is None:
        r_max = rows.shape[1] if rows is not None else ref.shape[0]
    dec = torch.empty((n_jobs, r_max, P), dtype=torch.float32, device=ref.device) if want_decision else None
    pred = torch.full((n_jobs, r_max), -1, dtype=torch.int32, device=ref.device)
    if kq is not None and kc is not None and kq.shape != kc.shape:
        raise ValueError("kq and kc differ in shape")
    _check(_lib().dk_svm_ovo_predict(ctx.handle, _ptr(kq), _ptr(kc), int(ref.stride(0)), int(ref.shape[0]),
                                     int(ref.shape[1]), n_jobs, _ptr(w),
                                     _ptr(rows), _ptr(row_count), int(r_max), _ptr(idx), _ptr(count), m_max,
                                     _ptr(coef), _ptr(bias), int(n_class), _ptr(dec), _ptr(pred), _stream(stream)),
           "dk_svm_ovo_predict")
    return {"decision": dec, "pred": pred}


def gram_stats(ctx: Context, kq: torch.Tensor | None, logkq: torch.Tensor | None = None,
               symmetric: bool = True, stream=None) -> dict:
    """dk_gram_stats: mean and variance of the off-diagonal K_q and log K_q of a Gram block
    (the strict upper triangle when symmetric), formed on the device. Reads back ten numbers."""
    ref = kq if kq is not None else logkq
    _need_cuda(kq, "kq", torch.float32)
    _need_cuda(logkq, "logkq", torch.float32)
    out = torch.empty(10, dtype=torch.float64, device=ref.device)
    _check(_lib().dk_gram_stats(ctx.handle, _ptr(kq), _ptr(logkq), int(ref.stride(0)), int(ref.shape[0]),
                                int(ref.shape[1]), 1 if symmetric else 0, _ptr(out), _stream(stream)),
           "dk_gram_stats")
    c, _, _, cl, _, _, kq_mean, kq_var, l_mean, l_var = out.cpu().tolist()
    res = {"pairs": int(c), "finite_log_pairs": int(cl)}
    if c > 0:
        res["kq_mean"], res["kq_var"] = kq_mean, kq_var
    if cl > 0:
        res["logkq_mean"], res["logkq_var"] = l_mean, l_var
    return res


def pca_fit(ctx: Context, x: torch.Tensor, k: int, sweeps: int = 10, stream=None) -> dict:
    """dk_pca_fit on the training rows x (m x p float32, CUDA): mean, scale, components
    (k x p), eigenvalues (k) and the remaining off-diagonal norm (a 1-element tensor)."""
    _need_cuda(x, "x", torch.float32)
    m, p = x.shape
    nbytes = int(_lib().dk_pca_workspace_bytes(int(p)))
    if nbytes == 0:
        raise ValueError(f"{p} features are outside the supported range")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    out = {"mean": torch.empty(p, dtype=torch.float32, device=x.device),
           "scale": torch.empty(p, dtype=torch.float32, device=x.device),
           "components": torch.empty((k, p), dtype=torch.float32, device=x.device),
           "eigenvalues": torch.empty(k, dtype=torch.float32, device=x.device),
           "off_norm": torch.empty(1, dtype=torch.float32, device=x.device)}
    _check(_lib().dk_pca_fit(ctx.handle, _ptr(x), int(m), int(p), int(k), int(sweeps), _ptr(ws), nbytes,
                             _ptr(out["mean"]), _ptr(out["scale"]), _ptr(out["components"]),
                             _ptr(out["eigenvalues"]), _ptr(out["off_norm"]), _stream(stream)), "dk_pca_fit")
    return out


def pca_transform(ctx: Context, x: torch.Tensor, model: dict, fit_range: bool, range_max: float = 3.141592653589793,
                  stream=None) -> torch.Tensor:
    """dk_pca_transform: m x k features in [0, range_max]. With fit_range the per-feature
    range is taken from these rows and stored in model["lo"] / model["hi"]; otherwise read."""
    _need_cuda(x, "x", torch.float32)
    m, p = x.shape
    k = model["components"].shape[0]
    if fit_range:
        model["lo"] = torch.empty(k, dtype=torch.float32, device=x.device)
        model["hi"] = torch.empty(k, dtype=torch.float32, device=x.device)
    out = torch.empty((m, k), dtype=torch.float32, device=x.device)
    _check(_lib().dk_pca_transform(ctx.handle, _ptr(x), int(m), int(p), _ptr(model["mean"]), _ptr(model["scale"]),
                                   _ptr(model["components"]), int(k), 1 if fit_range else 0, float(range_max),
                                   _ptr(model["lo"]), _ptr(model["hi"]), _ptr(out), _stream(stream)),
           "dk_pca_transform")
    return out
