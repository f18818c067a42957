"""The C-ABI library builds, loads and exports every symbol include/dualk.h declares.

CPU only: no kernel is launched. Calls made here either fail argument validation on
the host or find no device.
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dualk.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dk_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2602_01330_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("dk_mps_build", "dk_gram_tile", "dk_dual_kernel_rows"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} declared in dualk.h but not exported"


def test_binding_names_match_header():
    from paper_2602_01330_gb300 import dualk
    assert sorted(dualk.EXPORTED) == declared_symbols()


def test_only_dk_symbols_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2602_01330_gb300", "libdualk.so")],
                         capture_output=True, text=True).stdout
    names = [ln.split()[-1] for ln in out.splitlines() if ln.strip() and ln.split()[1] in ("T", "t")]
    assert names and all(n.startswith("dk_") for n in names if not n.startswith("_"))


def test_error_strings_and_host_validation(lib):
    lib.dk_error_string.restype = ctypes.c_char_p
    assert lib.dk_error_string(0) == b"ok"
    assert b"argument" in lib.dk_error_string(1)
    lib.dk_mps_bytes.restype = ctypes.c_size_t
    assert lib.dk_mps_bytes(10, 7, 4, 0) == 10 * 7 * 4 * 4 * 8     # chi^2 complex64 per sample-site
    assert lib.dk_mps_bytes(10, 7, 8, 1) == 10 * 7 * 8 * 8 * 16
    assert lib.dk_mps_bytes(0, 7, 4, 0) == 0
    # split-BF16 operands (DK_SPLIT_BF16 = 2): bond 32 only, 4 blocks x hi/lo x 16 rows of 40 BF16
    assert lib.dk_mps_bytes(10, 7, 32, 2) == 10 * 7 * 4 * 2 * 16 * 40 * 2
    assert lib.dk_mps_bytes(10, 7, 4, 2) == 0
    # no Gram-path call needs a workspace; unsupported combinations read as (size_t)-1
    lib.dk_workspace_bytes.restype = ctypes.c_size_t
    none = ctypes.c_size_t(-1).value
    for chi, dt, prec in ((4, 0, 0), (8, 0, 0), (32, 0, 0), (32, 0, 2), (4, 1, 1), (32, 2, 2)):
        assert lib.dk_workspace_bytes(784, chi, dt, prec) == 0
    for chi, dt, prec in ((16, 0, 0), (4, 0, 2), (8, 1, 1), (4, 1, 0), (32, 0, 1), (32, 2, 0), (8, 2, 2)):
        assert lib.dk_workspace_bytes(784, chi, dt, prec) == none
    assert lib.dk_workspace_bytes(0, 4, 0, 0) == none
    # block-state and PCA sizes
    lib.dk_block_states_bytes.restype = ctypes.c_size_t
    assert lib.dk_block_states_bytes(10, 784, 10) == 79 * 10 * 1024 * 8
    assert lib.dk_block_states_bytes(10, 20, 2) == 10 * 10 * 16 * 8   # dpad = 16 below 16 amplitudes
    assert lib.dk_block_states_bytes(10, 20, 13) == 0 and lib.dk_block_states_bytes(10, 20, 0) == 0
    # NULL context / pointers are rejected on the host before any CUDA call.
    assert lib.dk_mps_build(None, None, 1, 1, None, 0, None, None, None, None) == 1
    assert lib.dk_gram_tile(None, None, 1, None, 1, 1, 4, 0, 0, 1, 0, 1, None, None, None, None,
                            ctypes.c_float(1.0), ctypes.c_float(0.5), 0, None, None, None, None,
                            ctypes.c_int64(1), 0, None) == 1
    assert lib.dk_set_block_gram_form(None, 0) == 1  # DK_BLOCK_TCGEN05 on no context
    assert lib.dk_mps_split32(None, None, 1, 1, None, ctypes.c_size_t(0), None) == 1


def test_create_without_device_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is visible")
    h = ctypes.c_void_p()
    assert lib.dk_create(ctypes.byref(h), 0) == 6  # DK_ERR_NO_DEVICE


def test_workload_accounting():
    from paper_2602_01330_gb300 import workload
    assert workload.exact_bonds(6, 2) == [1, 2, 4, 4, 4, 2, 1]
    # dense count, n = 3: D = 1, 2, 2, 1 -> 16 (1*2 + 1*4) + 16 (4*2 + 2*4) + 16 (4*1 + 2*1) = 448
    assert workload.dense_flops_per_pair(3, 5) == 448
    # dense count, n = 784, reps = 2: 780 interior sites at D = 4 cost 2048 flops each
    edge = 16 * (1 * 2 + 1 * 4) + 16 * (4 * 4 + 2 * 16) + 16 * (16 * 2 + 4 * 4) + 16 * (4 * 1 + 2 * 1)
    assert workload.dense_flops_per_pair(784, 2) == 780 * 2048 + edge
    # block count, interior site at D = 4: 4 (s, t) terms of (2*2*2 + 2*2*2) complex MACs x 8
    assert workload.flops_per_pair(6, 2) - workload.flops_per_pair(5, 2) == 4 * 16 * 8
    # block count at n = 784: sites 1, 2, 783, 784 cost 32, 192, 192, 64 flops
    assert workload.flops_per_pair(784, 2) == 780 * 512 + 32 + 192 + 192 + 64
    assert workload.gram_entries(4) == 10 and workload.gram_entries(4, False, 3) == 12


def test_block_workspace_queries_without_context(lib):
    # The scratch queries of the block calls need a context (the plan depends on the SM
    # count); without one they return 0 rather than guess.
    lib.dk_block_states_workspace_bytes.restype = ctypes.c_size_t
    lib.dk_block_states_workspace_bytes.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4
    lib.dk_gram_blocks_workspace_bytes.restype = ctypes.c_size_t
    lib.dk_gram_blocks_workspace_bytes.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 7
    assert lib.dk_block_states_workspace_bytes(None, 100, 40, 10, 2) == 0
    assert lib.dk_gram_blocks_workspace_bytes(None, 40, 10, 100, 100, 2, 1, 1) == 0
