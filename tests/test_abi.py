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


def test_binding_constants_match_the_header(tmp_path):
    """Every constant the binding and the workload builder pass through the ABI
    (status codes and bits, precisions, solvers, field modes, circuits, node and
    cell kinds, diagnostic selectors and their device flag, the scalar count and
    the static solve's limit) has the header's value (the header compiled by the
    host C compiler prints its macros)."""
    import shutil
    import subprocess

    from paper_2310_04957_gb300 import pic
    from paper_2310_04957_gb300 import workloads as W

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    want = {
        "PIC_OK": pic.PIC_OK, "PIC_EINVAL": pic.PIC_EINVAL, "PIC_ENOMEM": pic.PIC_ENOMEM,
        "PIC_ECUDA": pic.PIC_ECUDA, "PIC_ENOCONV": pic.PIC_ENOCONV, "PIC_ETIMEOUT": pic.PIC_ETIMEOUT,
        "PIC_EOVERFLOW": pic.PIC_EOVERFLOW, "PIC_ENAN": pic.PIC_ENAN, "PIC_EIO": pic.PIC_EIO,
        "PIC_FLAG_OVERFLOW": pic.PIC_FLAG_OVERFLOW, "PIC_FLAG_TIMEOUT": pic.PIC_FLAG_TIMEOUT,
        "PIC_FLAG_NOCONV": pic.PIC_FLAG_NOCONV, "PIC_FLAG_NAN": pic.PIC_FLAG_NAN,
        "PIC_FP32": pic.PIC_FP32, "PIC_FP64": pic.PIC_FP64,
        "PIC_SOLVER_PLAIN": pic.PIC_SOLVER_PLAIN, "PIC_SOLVER_MIXED": pic.PIC_SOLVER_MIXED,
        "PIC_SOLVER_LEARNED": pic.PIC_SOLVER_LEARNED, "PIC_SOLVER_MG": pic.PIC_SOLVER_MG,
        "PIC_FIELD_DIRECT": pic.PIC_FIELD_DIRECT, "PIC_FIELD_VAHEDI": pic.PIC_FIELD_VAHEDI,
        "PIC_CIRCUIT_DIRECT": W.CIRCUIT_DIRECT, "PIC_CIRCUIT_RLC": W.CIRCUIT_RLC, "PIC_CIRCUIT_IMN": W.CIRCUIT_IMN,
        "PIC_NODE_FREE": W.NODE_FREE, "PIC_NODE_POWERED": W.NODE_POWERED, "PIC_NODE_GROUNDED": W.NODE_GROUNDED,
        "PIC_NODE_DRIVEN": W.NODE_DRIVEN, "PIC_CELL_PLASMA": W.CELL_PLASMA, "PIC_CELL_POWERED": W.CELL_POWERED,
        "PIC_CELL_GROUNDED": W.CELL_GROUNDED, "PIC_CELL_DIELECTRIC": W.CELL_DIELECTRIC,
        "PIC_DIAG_SCALARS": pic.DIAG_SCALARS, "PIC_DIAG_STORE": pic.DIAG_STORE,
        "PIC_DIAG_SOLVER": pic.DIAG_SOLVER, "PIC_DIAG_CIRCUIT": pic.DIAG_CIRCUIT,
        "PIC_DIAG_DEVICE": pic.DIAG_DEVICE, "PIC_NSCALARS": pic.NSCALARS,
        "PIC_STATIC_MAX_NODES": pic.STATIC_MAX_NODES,
        "PIC_DIAG_PHI": pic.DIAG["phi"], "PIC_DIAG_ER": pic.DIAG["Er"], "PIC_DIAG_EZ": pic.DIAG["Ez"],
        "PIC_DIAG_CHI": pic.DIAG["chi"], "PIC_DIAG_DEP_E": pic.DIAG["dep_e"], "PIC_DIAG_DEP_I": pic.DIAG["dep_i"],
        "PIC_DIAG_SIGMA": pic.DIAG["sigma"], "PIC_DIAG_VNODE": pic.DIAG["vnode"], "PIC_DIAG_RHO": pic.DIAG["rho"],
        "PIC_DIAG_NE_AVG": pic.DIAG["ne_avg"], "PIC_DIAG_NI_AVG": pic.DIAG["ni_avg"],
        "PIC_DIAG_PHI_WARM": pic.DIAG["phi_warm"], "PIC_DIAG_PHI_P": pic.DIAG["phiP"],
        "PIC_DIAG_PHI_L0": pic.DIAG["phiL0"],
    }
    names = sorted(want)
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "pic.h"\nint main(void) {\n' +
                   "\n".join(f'  printf("%lld\\n", (long long)({n}));' for n in names) + "\n  return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    bad = [(n, g, want[n]) for n, g in zip(names, got) if g != want[n]]
    assert not bad, bad
    assert [pic.DIAG[f"phiL{k}"] for k in range(4)] == [pic.DIAG["phiL0"] + k for k in range(4)]
