"""The C ABI without a GPU: libkf.so builds for sm_103a, loads, and exports every
function declared in include/kf.h; the ctypes structures match the header."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kf.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_1711_06571_gb300 import build
    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(kf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("kf_ctx_create", "kf_ctx_destroy", "kf_fit", "kf_make_seeds", "kf_bin_hits", "kf_build_besthit",
                 "kf_gather_hits", "kf_autotune_fit"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = C.CDLL(libpath)
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_binding_covers_every_symbol(libpath):
    from paper_1711_06571_gb300 import kf
    assert set(declared_functions()) == set(kf._SIGS)
    kf.load(libpath)
    assert "sm_103a" in kf.kf_version()


def test_struct_layouts_match_header(libpath, tmp_path):
    """Compile a tiny C program against include/kf.h that prints sizeof/offsetof of every
    struct, and compare with the ctypes mirror."""
    from paper_1711_06571_gb300 import kf
    structs = {
        "kf_surface": kf.kf_surface, "kf_geometry": kf.kf_geometry, "kf_fit_params": kf.kf_fit_params,
        "kf_seeds": kf.kf_seeds, "kf_track_hits": kf.kf_track_hits, "kf_tracks_out": kf.kf_tracks_out,
        "kf_binned_layer": kf.kf_binned_layer, "kf_build_params": kf.kf_build_params,
        "kf_server_params": kf.kf_server_params, "kf_event": kf.kf_event, "kf_event_result": kf.kf_event_result,
        "kf_server_stats": kf.kf_server_stats,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void){']
    for name, py in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for name, py in structs.items():
        assert int(got[name]) == C.sizeof(py), name
        for fname, _ in py._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(py, fname).offset, (name, fname)


def test_calls_fail_loudly_without_a_context(libpath):
    from paper_1711_06571_gb300 import kf
    L = kf.load(libpath)
    assert L.kf_fit(None, None, None, 0, None, None, None, None) == kf.KF_EINVAL
    assert L.kf_bin_hits(None, 0, None, None, None, 1.0, None, None, None, None) == kf.KF_EINVAL
    out = C.c_void_p()
    assert L.kf_server_create(None, None, None, C.byref(out)) == kf.KF_EINVAL
    assert L.kf_server_submit(None, None, None, None) == kf.KF_EINVAL
    assert L.kf_server_poll(None, 1, None) == kf.KF_EINVAL
    L.kf_server_destroy(None)
