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


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets
    (compiled with the host C compiler, no GPU needed)."""
    import subprocess
    from paper_2606_15924_gb300 import build
    build.build()
    from paper_2606_15924_gb300 import binding as B
    mirrors = {"tgs_camera": B.Camera, "tgs_gaussians": B.Gaussians, "tgs_param_ptrs": B.ParamPtrs,
               "tgs_projected": B.Projected, "tgs_sampling": B.Sampling, "tgs_loss_params": B.LossParams,
               "tgs_mlp": B.Mlp, "tgs_opt": B.Opt, "tgs_view_batch": B.ViewBatch,
               "tgs_density_params": B.DensityParams}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "turbogs.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        c, f, v = ln.split()
        got[(c, f)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
