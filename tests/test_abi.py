"""The C-ABI library loads and exports every function include/mpc3.h declares (no GPU needed:
nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mpc3.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = header_functions()
    for n in ("mpc_create", "mpc_share_input", "mpc_mult", "mpc_matmul", "mpc_verify_mult",
              "mpc_verify_matmul", "mpc_reconstruct", "mpc_ledger", "mpc_inject_fault"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2411_09287_gb300 import _lib, build
    if not os.path.exists(build.LIB):
        try:
            build.build()
        except RuntimeError as e:      # no toolkit on this host
            pytest.skip(str(e))
    lib = ctypes.CDLL(build.LIB)
    for name in header_functions():
        assert hasattr(lib, name), name
    assert set(header_functions()) == set(_lib.declared_symbols())


def test_binding_refuses_without_gpu_or_library(monkeypatch):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2411_09287_gb300 import mpc
    with pytest.raises(RuntimeError):
        mpc.Context(bytes(32))
