"""CPU checks of the boundary: libfw.so builds, loads without a GPU, and exports every
function include/fw.h declares (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

from paper_2205_03532_b300 import fw
from paper_2205_03532_b300.csrc import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fw_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(fw.ABI_FUNCTIONS)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_exports_nothing_else():
    out = subprocess.run(["nm", "-D", "--defined-only", B.build()], capture_output=True, text=True).stdout
    ours = {l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("fw_")}
    assert ours == set(_declared())


def test_config_defaults_without_gpu():
    cfg = fw.default_config()
    assert cfg.batch_size == 1024 and cfg.max_patches == 128 and cfg.patch_dirs == 6
    assert cfg.contact_gen == 0 and cfg.tri_iters == 16 and cfg.sdf_band == 0.0 and cfg.solver == 0
    assert abs(cfg.dt - 1 / 60) < 1e-7 and abs(cfg.gravity[2] + 9.81) < 1e-6
    assert abs(cfg.contact_offset - 1e-4) < 1e-9 and abs(cfg.cos_patch - 0.94) < 1e-7


def test_struct_layouts_match_header(tmp_path):
    assert ctypes.sizeof(fw.FwConfig) == 88   # 18 four-byte values (gravity has 3), a pointer, the seed
    # every field offset of the binding's fw_config against the C compiler's, from the header
    names = [f[0] for f in fw.FwConfig._fields_]
    src = tmp_path / "offsets.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"fw.h\"\nint main(void) {\n" +
                   "".join(f'  printf("%zu\\n", offsetof(fw_config, {n}));\n' for n in names) +
                   '  printf("%zu\\n", sizeof(fw_config));\n  return 0;\n}\n')
    exe = tmp_path / "offsets"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [getattr(fw.FwConfig, n).offset for n in names] + [ctypes.sizeof(fw.FwConfig)]
    assert got == want, (got, want)
    # the numpy record types the binding passes as arrays of fw_body_desc / fw_contact / fw_candidate
    from paper_2205_03532_b300 import scenes
    for ctype, dt in (("fw_body_desc", scenes.BODY_DTYPE), ("fw_contact", fw.CONTACT_DTYPE),
                      ("fw_candidate", fw.CANDIDATE_DTYPE)):
        src = tmp_path / f"{ctype}.c"
        src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"fw.h\"\nint main(void) {\n" +
                       "".join(f'  printf("%zu\\n", offsetof({ctype}, {n}));\n' for n in dt.names) +
                       f'  printf("%zu\\n", sizeof({ctype}));\n  return 0;\n}}\n')
        exe = tmp_path / ctype
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
        got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
        assert got == [dt.fields[n][1] for n in dt.names] + [dt.itemsize], (ctype, got)
    assert fw.CONTACT_DTYPE.itemsize == 52 and fw.CANDIDATE_DTYPE.itemsize == 32
