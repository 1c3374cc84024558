"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/pic.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pic.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pic_init", "pic_step", "pic_field_solve", "pic_diag", "pic_destroy", "pic_status"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2310_04957_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2310_04957_gb300 import pic

    assert sorted(pic.EXPORTS) == declared_functions()


def test_strerror_without_gpu():
    from paper_2310_04957_gb300 import build, pic

    build.build()
    assert pic.lib().pic_strerror(-4) == b"field solve did not converge within its iteration cap"
    assert pic.lib().pic_strerror(0) == b"ok"


def test_load_rejects_missing_and_foreign_files(tmp_path):
    """pic_load checks the file before it touches a GPU: a missing file and a
    file that is not a restart file both give PIC_EIO."""
    from paper_2310_04957_gb300 import build, pic

    build.build()
    h = ctypes.c_void_p()
    L = pic.lib()
    assert L.pic_load(str(tmp_path / "none").encode(), None, ctypes.byref(h)) == pic.PIC_EIO
    (tmp_path / "junk").write_bytes(b"not a restart file" * 10)
    assert L.pic_load(str(tmp_path / "junk").encode(), None, ctypes.byref(h)) == pic.PIC_EIO
    assert L.pic_strerror(pic.PIC_EIO).startswith(b"restart file")


@pytest.mark.parametrize("struct", ["Config", "Particles"])
def test_binding_structs_match_the_header(struct, tmp_path):
    """The binding's ctypes mirrors of pic_config and pic_particles have the
    header's field offsets and size (checked by compiling the header with the
    host C compiler)."""
    import shutil
    import subprocess

    from paper_2310_04957_gb300 import pic

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    py = getattr(pic, struct)
    cname = {"Config": "pic_config", "Particles": "pic_particles"}[struct]
    fields = [f[0] for f in py._fields_]
    lines = [f'  printf("%zu\\n", offsetof({cname}, {f}));' for f in fields]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "pic.h"\nint main(void) {\n' + "\n".join(lines) +
                   f'\n  printf("%zu\\n", sizeof({cname}));\n  return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [getattr(py, f).offset for f in fields] + [ctypes.sizeof(py)]
    assert got == want, list(zip(fields + ["sizeof"], got, want))
