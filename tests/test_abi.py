"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point include/*.h declares, and its structs match the ctypes layouts
of the binding.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1902_02999_gb300 import _abi, build as buildmod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(maclab_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound():
    lib = _abi.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(p[0] for p in _abi.PROTOTYPES) == names


def test_abi_version():
    assert _abi.load().maclab_abi_version() == 1


def test_create_rejects_bad_arguments_before_touching_a_gpu():
    lib = _abi.load()
    h = ctypes.c_void_p()
    g = _abi.Grid(0, 5, 1.0)
    p = _abi.Params()
    zb = (ctypes.c_double * 1)()
    m = (ctypes.c_uint8 * 1)()
    rc = lib.maclab_create(ctypes.byref(g), ctypes.byref(p), None, zb, m, None, None, None, None,
                           None, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert b"nx" in lib.maclab_last_error(None)
    assert lib.maclab_step(None, 1) == -1
    lib.maclab_destroy(None)


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "maclab.h"\n'
                   "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\","
                   "sizeof(maclab_grid),sizeof(maclab_params),sizeof(maclab_wave),"
                   "sizeof(maclab_bc),sizeof(maclab_allocator),sizeof(maclab_info),"
                   "offsetof(maclab_info,device_bytes),offsetof(maclab_params,h_ref));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(_abi.Grid), ctypes.sizeof(_abi.Params), ctypes.sizeof(_abi.Wave),
            ctypes.sizeof(_abi.BC), ctypes.sizeof(_abi.Allocator), ctypes.sizeof(_abi.Info),
            _abi.Info.device_bytes.offset, _abi.Params.h_ref.offset]
    assert got == want


def test_warm_start_config_layout_and_argument_checks(tmp_path):
    src = tmp_path / "ws.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "maclab_ws.h"\n'
                   "int main(void){printf(\"%zu %zu %zu %zu\\n\",sizeof(maclab_ws_config),"
                   "offsetof(maclab_ws_config,max_batch),offsetof(maclab_ws_config,seed),"
                   "offsetof(maclab_ws_config,tensor_path));return 0;}\n")
    exe = tmp_path / "ws"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(_abi.WSConfig), _abi.WSConfig.max_batch.offset, _abi.WSConfig.seed.offset,
                   _abi.WSConfig.tensor_path.offset]
    lib = _abi.load()
    cfg = _abi.WSConfig(res=48, channels=128, blocks=2, max_batch=1)   # res not a multiple of 64
    h = ctypes.c_void_p()
    assert lib.maclab_ws_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1 and not h.value
    assert b"multiples of 64" in lib.maclab_last_error(None)
    cfg = _abi.WSConfig(res=64, channels=128, blocks=2, max_batch=1, tensor_path=3)
    cfg.dilation[0] = cfg.dilation[1] = 1
    assert lib.maclab_ws_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1 and not h.value
    assert b"tensor_path" in lib.maclab_last_error(None)
    assert lib.maclab_ws_forward(None, 1, None, None) == -1


def test_build_targets_sm103a_only():
    assert buildmod.ARCH == "-gencode=arch=compute_103a,code=sm_103a"
    assert os.path.exists(buildmod.build())


def test_null_handles_are_argument_errors():
    """Every entry point that takes a handle answers a NULL one with
    MACLAB_E_ARG (no GPU involved)."""
    lib = _abi.load()
    c = ctypes.c_int()
    assert lib.maclab_autotune(None, 4, ctypes.byref(c)) == -1
    assert lib.maclab_set_temporal_block(None, 2) == -1
    assert lib.maclab_set_relaxation(None, 0.8) == -1
    assert lib.maclab_set_hbar_level(None, 1) == -1
    assert lib.maclab_set_graph_steps(None, 64) == -1
    assert lib.maclab_batch_step(None, 1) == -1
    assert lib.maclab_batch_set_graph_steps(None, 64) == -1
    assert lib.maclab_batch_set_persistent(None, 1) == -1
    assert b"NULL" in lib.maclab_batch_last_error(None)
    lib.maclab_batch_destroy(None)
