"""CPU checks of the C-ABI library: it builds, loads and exports every symbol
declared in include/blink.h.  No compute call is made (no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "blink.h")).read()
    return sorted(set(re.findall(r"BLINK_API\s+[\w\s\*]*?\b(blink_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_13478_gb300 import build, binding
    build.build()
    return binding.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("blink_grid", "blink_image_batch", "blink_cells", "blink_ctx_create",
                 "blink_plan_create", "blink_plan_image"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    for name in declared_symbols():
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr), name


def test_binding_lists_every_declared_symbol():
    from paper_2405_13478_gb300 import binding
    assert sorted(binding.EXPORTS) == declared_symbols()


def test_abi_version_and_sizes(lib):
    from paper_2405_13478_gb300 import binding
    assert lib.blink_abi_version() == 2
    sizes = binding.supported_sizes()
    for n in (128, 180, 256, 512, 1024):
        assert n in sizes
    assert all(n % 2 == 0 for n in sizes)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2405_13478_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            binding.lib(str(tmp_path / "nope.so"))
    finally:
        binding._lib = saved


def test_ctx_create_without_gpu_returns_error(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.blink_ctx_create(ctypes.byref(h), 0) != 0
    assert not h.value


def test_layer_array_matches_the_c_struct():
    import ctypes

    import numpy as np

    from paper_2405_13478_gb300 import binding
    arr = binding.layer_array([180, 256], [1, 0], [1.5e8, 1.6e8], [0.5, 0.25], [0, 32640],
                              [0, 32400])
    assert arr.itemsize == ctypes.sizeof(binding.Layer) == 40
    p = binding.make_layers(arr)
    assert p[1].n_px == 256 and p[1].weighting == 0 and p[1].freq_hz == 1.6e8
    assert p[1].delta_u == 0.25 and p[1].vis_offset == 32640 and p[1].out_offset == 32400
    d = binding.make_layers([dict(n_px=180, weighting=1, freq_hz=1.5e8, delta_u=0.5,
                                  vis_offset=0, out_offset=0)])
    assert bytes(d[0]) == np.asarray(arr[0:1]).tobytes()


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Field offsets and sizes of blink_layer and blink_epilogue as the C
    compiler lays them out from include/blink.h, against the ctypes mirrors."""
    import ctypes
    import os
    import shutil
    import subprocess

    from paper_2405_13478_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    fields = {"blink_layer": [f for f, _ in binding.Layer._fields_],
              "blink_epilogue": [f for f, _ in binding.Epilogue._fields_]}
    lines = ["#include <stdio.h>", "#include \"blink.h\"", "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st, cls in (("blink_layer", binding.Layer), ("blink_epilogue", binding.Epilogue)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
