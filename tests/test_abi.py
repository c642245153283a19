"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/mcrt.h declares.  No compute call is made."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mcrt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcrt_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_1902_01137_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["mcrt_create", "mcrt_destroy", "mcrt_scene_create", "mcrt_scene_build_majorants",
              "mcrt_scene_read_majorants", "mcrt_trace_camera", "mcrt_trace_flux", "mcrt_tally_read",
              "mcrt_tally_destroy", "mcrt_scene_destroy", "mcrt_debug_dda", "mcrt_status_string",
              "mcrt_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_exports_nothing_else(built):
    # hidden visibility: only the C entry points are dynamic symbols
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    ours = sorted({l.split()[-1] for l in out.splitlines() if " T " in l and "mcrt" in l})
    assert set(ours) <= set(declared_functions()), set(ours) - set(declared_functions())


def test_binding_argument_checks_without_gpu(built):
    import paper_1902_01137_gb300 as m
    L = m.lib()
    assert L.mcrt_status_string(m.MCRT_ERR_ARG) == b"invalid argument"
    assert L.mcrt_create(None, 0, None) == m.MCRT_ERR_ARG
    assert L.mcrt_scene_create(None, None, None) == m.MCRT_ERR_ARG
    assert L.mcrt_trace_flux(None, 1, 0, None, None) == m.MCRT_ERR_ARG
    assert L.mcrt_tally_read(None, None, None, None, 0) == m.MCRT_ERR_ARG
    o = m.mcrt_trace_opts_default()
    assert o.tau_merge == 1.0 and o.finest_level == 0 and o.sun_mode == m.MCRT_SUN_RATIO
    assert o.schedule == m.MCRT_SCHEDULE_PERSISTENT and o.wavefront_slots == 0
    v = C.c_int32()
    assert L.mcrt_version(C.byref(v)) == 0 and v.value == m.ABI_VERSION


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures have the C structures' sizes and field offsets
    (gcc compiles a probe against include/mcrt.h)."""
    import shutil
    import subprocess
    import paper_1902_01137_gb300 as m
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    structs = {"mcrt_trace_opts": m.TraceOpts, "mcrt_camera_desc": m.CameraDesc,
               "mcrt_field_desc": m.FieldDesc, "mcrt_batch_item": m.BatchItem}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcrt.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[cname + "." + f]) == getattr(py, f).offset, (cname, f)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_1902_01137_gb300 as m
    monkeypatch.setattr(m, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(m, "_lib", None)
    with pytest.raises(ImportError):
        m.lib()
