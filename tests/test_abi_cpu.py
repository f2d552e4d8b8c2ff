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
