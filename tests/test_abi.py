"""The C-ABI library builds for sm_103a, loads, and exports every function include/rgs.h
declares; the ctypes mirrors of the header's structs have the C layout. No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2601_00705_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rgs.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rgs_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert sorted(binding.EXPORTED) == _declared_functions()


def test_library_builds_loads_and_exports_every_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_ctypes_structs_match_c_layout(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rgs.h"\n'
                   "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
                   "sizeof(rgs_gaussians), sizeof(rgs_camera), sizeof(rgs_config),"
                   "sizeof(rgs_images), sizeof(rgs_image_grads), sizeof(rgs_stats),"
                   "offsetof(rgs_config, tile_w), sizeof(rgs_track_config),"
                   "sizeof(rgs_adam_config), offsetof(rgs_adam_config, iterations),"
                   "sizeof(rgs_seed_config), sizeof(rgs_map_reg), sizeof(rgs_prune_config),"
                   "offsetof(rgs_config, sh_ready_event));"
                   "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                            check=True).stdout.split()]
    assert sizes == [ctypes.sizeof(binding.Gaussians), ctypes.sizeof(binding.Camera),
                     ctypes.sizeof(binding.Config), ctypes.sizeof(binding.Images),
                     ctypes.sizeof(binding.ImageGrads), ctypes.sizeof(binding.Stats),
                     binding.Config.tile_w.offset, ctypes.sizeof(binding.TrackConfig),
                     ctypes.sizeof(binding.AdamConfig), binding.AdamConfig.iterations.offset,
                     ctypes.sizeof(binding.SeedConfig), ctypes.sizeof(binding.MapReg),
                     ctypes.sizeof(binding.PruneConfig), binding.Config.sh_ready_event.offset]


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = binding.load()
    h = ctypes.c_void_p()
    assert lib.rgs_create(ctypes.byref(h), 0) == binding.RGS_ERR_INVALID_ARG
    assert lib.rgs_create(None, 0) == binding.RGS_ERR_INVALID_ARG


def test_single_pass_scan_sizes_and_refuses_bad_arguments_before_any_gpu_work():
    lib = binding.load()
    # Work area: a 16-byte header, then one 8-byte state per tile of 4096 elements, plus two
    # (the bound the bitmask compaction also fits in).
    for n in (0, 1, 4095, 4096, 4097, 1 << 20):
        assert lib.rgs_single_pass_scan_bytes(n) == 16 + 8 * ((n + 4095) // 4096 + 2), n
    assert lib.rgs_single_pass_scan_bytes(-1) == 0
    p = ctypes.c_void_p
    fake = 1 << 20  # never dereferenced: every call below returns before any GPU work
    need = lib.rgs_single_pass_scan_bytes(4096)

    def call(n, inp=fake, work=fake, nbytes=need, status=fake):
        return lib.rgs_exclusive_scan_u32_single_pass(p(inp), p(fake), n, None, p(work), nbytes,
                                                      p(status), None)

    bad = binding.RGS_ERR_INVALID_ARG
    assert call(-1) == bad
    assert call(1 << 31) == bad
    assert call(4096, nbytes=need - 8) == bad
    assert call(4096, work=fake + 8) == bad  # not 16-byte aligned
    assert call(4096, work=None) == bad
    assert call(4096, status=None) == bad
    assert call(4096, inp=None) == bad
    # Nothing to scan and no total to write: nothing runs.
    assert call(0, inp=None) == binding.RGS_OK
