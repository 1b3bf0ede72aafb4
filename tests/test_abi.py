"""The C-ABI library builds, loads without a GPU, and exports every entry
point include/turbogs.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "turbogs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tgs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for call in ("select_tiles", "project_gaussians", "bin_tiles", "render_sampled", "loss_sparse_ncc",
                 "backward_sampled", "hybrid_step"):
        assert "tgs_" + call in names


def test_library_exports_every_declared_symbol():
    from paper_2606_15924_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.tgs_version.restype = ctypes.c_char_p
    assert lib.tgs_version().startswith(b"turbogs-gb300")


def test_binding_names_match_the_abi():
    from paper_2606_15924_gb300 import build
    build.build()
    from paper_2606_15924_gb300 import binding
    for n in _declared():
        assert n in binding.EXPORTED
        short = n[len("tgs_"):]
        if short not in ("version", "last_cuda_error", "status_string", "device_check"):
            assert hasattr(binding, short), short
