"""CPU-only checks of the C ABI library: it builds for sm_103a, loads, and
exports every function include/pplbm.h declares.  No GPU work is done."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "pplbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(lbm_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_07968_gb300 import build

    return ctypes.CDLL(build.build())


def test_library_exports_every_declared_function(lib):
    names = header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_function():
    from paper_2003_07968_gb300 import capi

    assert sorted(capi.SIGNATURES) == header_functions()


def test_struct_layouts_match_header(lib, tmp_path):
    # sizes of the ctypes mirrors against a tiny C program compiled with the header
    from paper_2003_07968_gb300 import capi

    src = ('#include "pplbm.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(){printf("%zu %zu %zu %zu %zu %zu %zu\\n",'
           'sizeof(lbm_lattice_desc), sizeof(lbm_runtime_opts), sizeof(lbm_kernel_stat),'
           'sizeof(lbm_info_t), offsetof(lbm_lattice_desc, mrt_rates), sizeof(lbm_server_opts),'
           'sizeof(lbm_server_stats));return 0;}')
    c = str(tmp_path / "layout.c")
    exe = str(tmp_path / "layout")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(capi.LatticeDesc), ctypes.sizeof(capi.RuntimeOpts),
            ctypes.sizeof(capi.KernelStat), ctypes.sizeof(capi.Info),
            capi.LatticeDesc.mrt_rates.offset, ctypes.sizeof(capi.ServerOpts),
            ctypes.sizeof(capi.ServerStats)]
    assert got == want


def test_strerror_and_defaults_without_gpu():
    from paper_2003_07968_gb300 import capi

    assert "psi" in capi.lbm_strerror(capi.LBM_ERR_NUMERIC)
    d = capi.lbm_desc_default(64, 32)
    assert (d.nx, d.ny, d.tau, d.G, d.eps, d.sigma) == (64, 32, 1.0, -1.0, 1.73, 1.0)
    assert d.eos_a == 3.852462257 and d.eos_k == 0.01


def test_missing_library_fails_loudly(tmp_path):
    from paper_2003_07968_gb300 import capi

    with pytest.raises(ImportError):
        capi._lib_backup = capi._lib
        capi._lib = None
        try:
            capi.load(str(tmp_path / "nope.so"))
        finally:
            capi._lib = capi._lib_backup


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2003_07968_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "pplbm_oracle" not in txt, f


def test_staging_copy_plans_are_proven_on_the_host():
    # every bulk copy the TMA passes issue is 16-byte aligned on both sides,
    # a multiple of 16 bytes long, inside its allocation and box, and the
    # copies cover every value an active site reads (no GPU involved)
    from paper_2003_07968_gb300 import capi

    rc, report = capi.lbm_selfcheck()
    assert rc == 0, report
    assert report.startswith("ok:")
