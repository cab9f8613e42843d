"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and the host-only entry points agree with the paper's storage
counts (Sec. 3.2.3, Sec. 4, Sec. 5.3).  No compute call is made (no GPU)."""
import ctypes as C
import os
import subprocess

import pytest

from paper_1511_07226_gb300 import pfk


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pfk.LIB_PATH):
        from paper_1511_07226_gb300 import build
        build.build()
    return pfk.load()


def test_every_header_symbol_is_exported(lib):
    names = pfk.header_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", pfk.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_abi_version(lib):
    assert lib.pfk_abi_version() == 1


@pytest.mark.parametrize("method,mmax,count", [
    ("pipefcg", 30, 4 * 30 + 11), ("fcg", 30, 30 + 6), ("gcr", 30, 2 * 30 + 7),
    ("pipegcr", 30, 2 * 30 + 7 + 30 + 2), ("fgmres", 30, 2 * 30 + 2), ("pipefgmres", 30, 4 * 30 + 2),
    ("pipefcg", 1, 15), ("pipegcr_w", 30, 4 * 30 + 11)])
def test_storage_vector_counts_follow_paper(lib, method, mmax, count):
    assert pfk.storage_vectors(method, mmax) == count


def test_workspace_accounts_rings(lib):
    n = 1000
    b = pfk.workspace_bytes("pipefcg", 30, n)
    # x is the caller's; the library keeps the other vectors of the paper's count
    # (r, u, w, m, n, p/s/q/z rings of nu+1) plus t = w - r and one scratch vector
    assert b == (7 + 4 * 31) * n * 8


def test_default_params(lib):
    p = pfk.default_params()
    assert p.method == pfk.METHODS["pipefcg"] and p.mmax == 30 and p.rtol == 1e-8
    assert p.true_residual_check == 1 and p.graph_iters == 8


def test_invalid_arguments_rejected_without_gpu(lib):
    out = C.c_int64()
    assert lib.pfk_solve_workspace_bytes(1, 0, 10, C.byref(out)) == -1
    assert lib.pfk_solve_workspace_bytes(1, 33, 10, C.byref(out)) == -1
    assert lib.pfk_method_storage_vectors(99, 3) == -1
    assert lib.pfk_create_context(0, None, None) == -1
    assert b"NULL" in lib.pfk_last_error(None)


def test_struct_layouts():
    assert C.sizeof(pfk.OperatorDesc) == 112
    assert C.sizeof(pfk.PcDesc) == 32
    assert C.sizeof(pfk.SolveParams) == 80
    assert C.sizeof(pfk.SolveInfo) == 96


def _ctypes_layouts():
    structs = {"pfk_operator_desc": pfk.OperatorDesc, "pfk_pc_desc": pfk.PcDesc,
               "pfk_solve_params": pfk.SolveParams, "pfk_solve_info": pfk.SolveInfo,
               "pfk_server_params": pfk.ServerParams, "pfk_request": pfk.Request}
    return structs


def test_struct_layouts_match_c_header(tmp_path):
    """Every ctypes structure has the size and field offsets the C compiler gives
    the header's structure."""
    structs = _ctypes_layouts()
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{pfk.HEADER}"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line)
    for cname, cls in structs.items():
        assert int(got[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_storage_counts_match_the_paper_golden_file(lib):
    """tests/golden/storage_counts.txt holds the paper's stated vector counts."""
    path = os.path.join(os.path.dirname(__file__), "golden", "storage_counts.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 7
    for method, a, b, *_ in rows:
        for nu in (1, 5, 30, 32):
            assert pfk.storage_vectors(method, nu) == int(a) * nu + int(b), (method, nu)


def test_inner_solve_struct_layout(tmp_path):
    src = tmp_path / "inner.c"
    src.write_text(f'#include <stdio.h>\n#include <stddef.h>\n#include "{pfk.HEADER}"\n'
                   'int main(void) { printf("%zu %zu %zu %zu\\n", sizeof(pfk_inner_solve), '
                   'offsetof(pfk_inner_solve, rtol), offsetof(pfk_inner_solve, maxit), '
                   'offsetof(pfk_inner_solve, pad)); return 0; }')
    exe = tmp_path / "inner"
    subprocess.run(["gcc", "-std=c11", str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [C.sizeof(pfk.InnerSolve), pfk.InnerSolve.rtol.offset, pfk.InnerSolve.maxit.offset,
                   pfk.InnerSolve.pad.offset]
