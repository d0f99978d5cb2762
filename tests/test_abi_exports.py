"""The C-ABI library builds for sm_103a and exports every function that
include/nswe.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(nswe_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for call in ["nswe_residual", "nswe_jacobian_simplified", "nswe_jacobian_full", "nswe_mg_vcycle",
                 "nswe_newton_solve"]:
        assert call in names


def test_library_exports_every_declared_symbol():
    from paper_2505_10857_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2505_10857_gb300 import nswe
    assert set(declared_functions()) <= set(nswe.EXPORTS)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2505_10857_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "from oracle" not in src and "nswe_oracle" not in src, fn


def test_binding_structs_match_the_header(tmp_path):
    """Field offsets and sizes of nswe_params / nswe_info / nswe_bc1d as the
    C compiler lays them out agree with the ctypes mirrors."""
    import subprocess
    from paper_2505_10857_gb300 import nswe
    structs = {"nswe_params": nswe.Params, "nswe_info": nswe.Info, "nswe_bc1d": nswe.BC1D,
               "nswe_server_config": nswe.ServerConfig, "nswe_server_times": nswe.ServerTimes,
               "nswe_server_stats": nswe.ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nswe.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_solve_shapes_listed():
    from paper_2505_10857_gb300 import nswe
    shapes = nswe.solve_shapes()
    assert shapes[0] == (256, 4) and len(shapes) >= 2
    for t, b in shapes:
        assert t % 32 == 0 and t * b <= 2048 and t * b * 64 <= 65536 * 2


def _fake_problem(cls, levels, dims):
    """A binding problem object without a device-side problem: only the
    sizes the host-side checks read."""
    import ctypes as _ct
    p = object.__new__(cls)
    p.h = _ct.c_void_p()  # no handle: close() does nothing
    p.levels = levels
    if cls.__name__ == "Problem2D":
        p.Nx, p.Ny = dims
        p.cells = lambda l=0: (p.Nx >> l) * (p.Ny >> l)
    else:
        p.N = dims
        p.cells = lambda l=0: p.N >> l
    return p


def test_binding_refuses_arrays_smaller_than_their_level():
    """The per-level calls take bare pointers in C, so the binding checks the
    sizes first: U, R, dU [comps][n_l] and J [nb][comps^2][n_l]. A level or
    nb the C call does not accept is left to the C call to refuse."""
    import pytest
    torch = pytest.importorskip("torch")
    from paper_2505_10857_gb300 import nswe
    chk = nswe._check_level_sizes
    p2 = _fake_problem(nswe.Problem2D, 3, (32, 16))
    n0, n2 = 32 * 16, 8 * 4
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64)
    chk("call", p2, 0, 9, U=z(3, n0), R=z(3, n0), J=z(9, 9, n0))
    chk("call", p2, 2, 21, U=z(3, n2), R=z(3, n2), J=z(21, 9, n2), dU=z(3, n2))
    chk("call", p2, 0, 9, U=z(3, n0 * 2))  # larger is fine
    for bad in (dict(U=z(3, n2)), dict(R=z(3, n0 - 1)), dict(dU=z(2, n0)), dict(J=z(9, 9, n0 // 4))):
        with pytest.raises(ValueError):
            chk("call", p2, 0, 9, **bad)
    with pytest.raises(ValueError):
        chk("call", p2, 0, 21, J=z(9, 9, n0))  # J9-sized array for J21
    chk("call", p2, 3, 9, U=z(1))      # level outside 0..2: the C call refuses it
    chk("call", p2, 0, 7, J=z(1))      # nb 7: the C call refuses it
    chk("call", p2, 0, 9, U=None, R=12345)  # no array, or a raw pointer: not checked
    p1 = _fake_problem(nswe.Problem1D, 4, 200)
    chk("call", p1, 1, 3, U=z(2, 100), R=z(2, 100), J=z(3, 4, 100))
    with pytest.raises(ValueError):
        chk("call", p1, 0, 5, J=z(3, 4, 200))
    with pytest.raises(ValueError):
        chk("call", p1, 0, 3, U=z(3, 100))
    chk("call", p1, 0, 9, J=z(1))      # a 2D nb on a 1D problem: the C call refuses it
