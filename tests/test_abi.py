"""The C-ABI library builds, loads and exports every entry point include/adr.h
declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2409_08669_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(adr_[a-z_0-9]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    try:
        return build.build()
    except RuntimeError as e:
        pytest.fail(f"libadr.so did not build: {e}")


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("adr_create", "adr_destroy", "adr_preprocess", "adr_sort", "adr_render",
                     "adr_num_pairs", "adr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_covers_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name)
    assert declared_functions() <= set(_lib.exported_names())


def test_struct_layouts_match_header():
    assert ctypes.sizeof(_lib.adr_camera) == (16 + 4 + 1 + 3) * 4 + 2 * 4
    assert ctypes.sizeof(_lib.adr_settings) == 4 + 4 * 4 + 3 * 4 + 4 + 4 + 4
    assert ctypes.sizeof(_lib.adr_serve_config) == 8 + 3 * 8 + 5 * 4 + 4   # + tail padding


def test_version_and_error_without_gpu(libpath):
    lib = _lib.load()
    assert lib.adr_version().startswith(b"adr-gb300")
    # invalid arguments are rejected before any CUDA call
    out = ctypes.c_void_p()
    st = lib.adr_create(ctypes.byref(out), 0, 10, 16, 16, 0)
    assert st == _lib.ADR_ERR_INVALID
    assert b"max_gaussians" in lib.adr_last_error()


def test_scene_size_limit_rejected_without_gpu(libpath):
    # the per-Gaussian kernels index 4 * i + c in 32 bits: 2^29 is the largest scene
    lib = _lib.load()
    out = ctypes.c_void_p()
    for n in ((1 << 29) + 1, 1 << 30, 1 << 40):
        assert lib.adr_create(ctypes.byref(out), n, 1 << 20, 64, 64, 0) == _lib.ADR_ERR_INVALID
        assert b"2^29" in lib.adr_last_error()
        assert not out.value
    cfg = _lib.adr_serve_config(max_slots=1, mem_budget_bytes=1 << 30, slot_pair_capacity=1 << 20,
                                slot_max_gaussians=(1 << 29) + 1, max_width=256, max_height=256,
                                use_graphs=1, device=0, max_batch=1)
    assert lib.adr_serve_create(ctypes.byref(out), ctypes.byref(cfg)) == _lib.ADR_ERR_INVALID
    assert not out.value


def test_serve_config_rejected_without_gpu(libpath):
    lib = _lib.load()
    cfg = _lib.adr_serve_config(max_slots=0, mem_budget_bytes=1 << 30, slot_pair_capacity=1 << 20,
                                slot_max_gaussians=1 << 16, max_width=256, max_height=256,
                                use_graphs=1, device=0, max_batch=1)
    out = ctypes.c_void_p()
    assert lib.adr_serve_create(ctypes.byref(out), ctypes.byref(cfg)) == _lib.ADR_ERR_INVALID
    assert not out.value
    cfg.max_slots, cfg.max_width = 2, 8192
    assert lib.adr_serve_create(ctypes.byref(out), ctypes.byref(cfg)) == _lib.ADR_ERR_INVALID
    # batches of 1..4 requests, the slots a whole number of batch groups
    cfg.max_width = 256
    for slots, batch in ((4, 0), (8, 5), (6, 4), (3, 2)):
        cfg.max_slots, cfg.max_batch = slots, batch
        assert lib.adr_serve_create(ctypes.byref(out), ctypes.byref(cfg)) == _lib.ADR_ERR_INVALID
        assert not out.value
    assert lib.adr_serve_poll(None, 1, 0) == _lib.ADR_ERR_INVALID


def test_settings_marshalling_carries_every_field():
    from paper_2409_08669_gb300 import scenes as S
    st = S.Settings(mode=S.MODE_CIRCLE, alpha_low=float(np.float32(2 / 255)), t_min=1e-3,
                    lowpass=0.2, jac_clamp=1.1, bg=(0.1, 0.2, 0.3), sh_degree=2,
                    rect_rule=S.RECT_3DGS, load_grad=S.LOAD_GRAD_TERMINATION)
    c = _lib.make_settings(st)
    assert (c.mode, c.sh_degree, c.rect_rule, c.load_grad) == (1, 2, 1, 1)
    assert c.alpha_low == pytest.approx(2 / 255, rel=1e-6) and c.t_min == pytest.approx(1e-3)
    assert (c.lowpass, c.jac_clamp) == (pytest.approx(0.2), pytest.approx(1.1))
    assert list(c.bg) == [pytest.approx(0.1), pytest.approx(0.2), pytest.approx(0.3)]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without libadr.so the binding raises instead of computing
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib._build, "LIB", str(tmp_path / "libadr.so"))
    with pytest.raises(RuntimeError, match="libadr.so not found"):
        _lib.load(build_if_missing=False)


def test_parameter_checks_reject_what_the_kernels_would_overrun():
    # the binding's checks run before any C call: sizes, dtypes and layout
    import torch
    from paper_2409_08669_gb300.raster import check_params, check_tensor
    n = 5
    good = [torch.zeros(n, 3), torch.ones(n, 3), torch.ones(n, 4), torch.ones(n), torch.zeros(n, 16, 3)]
    assert check_params(good) == n
    assert check_params([torch.zeros(0, 3), torch.zeros(0, 3), torch.zeros(0, 4), torch.zeros(0),
                         torch.zeros(0, 16, 3)]) == 0
    bad_sh = good[:4] + [torch.zeros(n, 9, 3)]            # degree-2 SH: 27 values, not 48
    with pytest.raises(ValueError, match="sh holds 135 values, expected 240"):
        check_params(bad_sh)
    with pytest.raises(ValueError, match="float32"):
        check_params(good[:3] + [torch.ones(n, dtype=torch.float64)] + good[4:])
    with pytest.raises(ValueError, match="contiguous"):
        check_params([torch.zeros(3, n).t()] + good[1:])
    with pytest.raises(ValueError, match=r"\[n, 3\]"):
        check_params([torch.zeros(3 * n)] + good[1:])
    with pytest.raises(ValueError, match="expected 5"):
        check_params(good[:4])
    with pytest.raises(ValueError, match="must be on cuda:0"):
        check_params(good, device=0)                      # CPU tensors
    with pytest.raises(ValueError, match="int32"):
        check_tensor("load", torch.zeros(4), 4, dtype=torch.int32)
    with pytest.raises(TypeError):
        check_tensor("img", np.zeros(4, np.float32), 4)


def test_serving_request_image_checked_before_submit():
    import torch
    from paper_2409_08669_gb300 import scenes as S
    from paper_2409_08669_gb300.serve import Server
    srv = Server.__new__(Server)          # no server: only the binding's checks run
    srv.device, srv._h = 0, None
    cam = S.look_at((0, 0, -3), width=32, height=24)
    with pytest.raises(ValueError, match=r"\[3, 24, 32\]"):
        srv._check_out(cam, torch.empty(3, 32, 24))
    with pytest.raises(ValueError, match="cuda:0"):
        srv._check_out(cam, torch.empty(3, 24, 32))
    with pytest.raises(ValueError, match="expected 5 parameter tensors"):
        srv.add_scene([torch.zeros(1, 3)], S.Settings())


def test_product_path_never_touches_the_oracle():
    # the package and its CUDA sources name neither the oracle package nor its library
    pkg = os.path.join(ROOT, "paper_2409_08669_gb300")
    offenders = []
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for fn in files:
            if not fn.endswith((".py", ".cu", ".cuh", ".h")):
                continue
            text = open(os.path.join(dirpath, fn)).read()
            if re.search(r"^\s*(import oracle|from oracle\b)|liboracle|adr_oracle", text, re.M):
                offenders.append(os.path.relpath(os.path.join(dirpath, fn), ROOT))
    assert not offenders, offenders


def test_oracle_never_touches_the_product():
    # the oracle imports nothing from the package and includes none of its headers
    odir = os.path.join(ROOT, "oracle")
    for fn in os.listdir(odir):
        if fn.endswith((".py", ".c", ".h")):
            text = open(os.path.join(odir, fn)).read()
            assert not re.search(r"paper_2409_08669_gb300|adr_internal|libadr|include/adr", text), fn


def test_lookback_expiry_hook_checks_its_arguments_without_gpu(libpath):
    lib = _lib.load()
    assert lib.adr_test_lookback_expiry(0, 0) == _lib.ADR_ERR_INVALID
    assert lib.adr_test_lookback_expiry(1, (1 << 22) + 1) == _lib.ADR_ERR_INVALID
    assert b"spin_limit" in lib.adr_last_error()
    assert lib.adr_test_lookback_expiry(-1, 0) == _lib.ADR_OK


_STATUS_MAP_SRC = r"""
#include <cstdio>
#include "status_bits.h"
int main() {
    for (unsigned bits = 0; bits < 8; ++bits)
        for (int over = 0; over < 2; ++over) {
            const adr::StatusReport r = adr::status_from_bits(bits, over ? 11 : 10, 10);
            std::printf("%u %d %d %d\n", bits, over, (int)r.status, r.message[0] != 0);
        }
    return 0;
}
"""


def test_device_status_word_maps_to_one_status_in_every_entry_point(tmp_path):
    """The mapping adr_sync_status, adr_render_frame_noalloc and the serving
    scheduler share (host code, compiled here with g++): a wait that gave up
    wins (its frame reads as saturated), then a pair overflow (flag or count
    above the capacity), then a failed consistency check; every error has a
    message."""
    src = tmp_path / "status_map.cpp"
    exe = tmp_path / "status_map"
    src.write_text(_STATUS_MAP_SRC)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run(["g++", "-std=c++17", f"-I{os.path.join(root, 'include')}",
                    f"-I{os.path.join(root, 'paper_2409_08669_gb300', 'csrc')}", str(src), "-o", str(exe)],
                   check=True)
    rows = [tuple(map(int, line.split())) for line in
            subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()]
    assert len(rows) == 16
    for bits, over, status, has_msg in rows:
        if bits & 2:
            want = _lib.ADR_ERR_TIMEOUT
        elif (bits & 1) or over:
            want = _lib.ADR_ERR_CAPACITY
        elif bits & 4:
            want = _lib.ADR_ERR_CUDA
        else:
            want = _lib.ADR_OK
        assert status == want, (bits, over, status)
        assert has_msg == (want != _lib.ADR_OK)
