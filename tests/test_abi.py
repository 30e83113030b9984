"""The C ABI: the library builds for sm_103a, loads, exports every function
declared in include/reed.h, and the Python structs match the C layout.
No compute calls are made (no GPU needed)."""
import os
import re
import subprocess
import ctypes

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "reed.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(reed_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libreed():
    from paper_0810_4737_gb300 import build as B
    B.build()
    return ctypes.CDLL(B.LIB)


def test_library_exports_every_declared_symbol(libreed):
    names = _declared()
    assert "reed_init" in names and "reed_run" in names and "reed_range_profile" in names
    for n in names:
        assert hasattr(libreed, n), n
    from paper_0810_4737_gb300 import reed as R
    assert sorted(R.EXPORTED) == names


def test_struct_layouts_match_the_header(tmp_path):
    from paper_0810_4737_gb300 import reed as R
    structs = ["reed_lattice", "reed_species", "reed_potentials", "reed_run_opts", "reed_track_record",
               "reed_stats_t"]
    prog = tmp_path / "sz.c"
    body = "".join('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (s, s) for s in structs)
    prog.write_text('#include <stdio.h>\n#include "reed.h"\nint main(void){%s return 0;}\n' % body)
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = dict(zip(out[0::2], map(int, out[1::2])))
    for s in structs:
        assert ctypes.sizeof(getattr(R, s)) == sizes[s], s
    assert R.RECORD_DTYPE.itemsize == sizes["reed_track_record"]


def test_library_is_built_for_sm103a():
    from paper_0810_4737_gb300 import build as B
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
    B.build()
    out = subprocess.run(["cuobjdump", "--list-elf", B.LIB], capture_output=True, text=True)
    if out.returncode == 0:
        assert "sm_103" in out.stdout


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_0810_4737_gb300 import reed as R
    monkeypatch.setattr(R, "_LIB", None)
    monkeypatch.setattr(R, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        R.lib()


def test_binding_constants_match_the_header():
    from paper_0810_4737_gb300 import reed as R
    src = open(os.path.join(ROOT, "include", "reed.h")).read()
    d = {k: int(v) for k, v in re.findall(r"#define REED_([A-Z0-9_]+)\s+(-?\d+)", src)}
    for name in ("OK", "E_ARG", "E_CUDA", "E_TIMEOUT", "E_QUEUE_FULL", "E_NONFINITE", "E_NOMEM", "E_SMEM",
                 "E_STATE", "E_NEIGHBOR", "PREC_MIXED", "PREC_FP64"):
        assert getattr(R, name) == d[name], name
    for table, prefix in ((R.LATTICE, "LATTICE_"), (R.TT, "TT_"), (R.BEAM, "BEAM_"), (R.TARGET, "TARGET_")):
        declared = {k[len(prefix):].lower(): v for k, v in d.items() if k.startswith(prefix)}
        assert table == declared, prefix
    assert (R.STOPPED, R.BACKSCATTERED, R.TRUNCATED, R.FAILED) == tuple(
        d["TRACK_" + k] for k in ("STOPPED", "BACKSCATTERED", "TRUNCATED", "FAILED"))
