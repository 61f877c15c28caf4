"""The C-ABI library builds, loads and exports every entry point that
include/o2pic.h declares; host-side validation works without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_0705_0495_gb300 import build, inputs, o2pic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(pic_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return o2pic.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pic_init" in names and "pic_step" in names and "pic_diagnostics" in names
    raw = C.CDLL(o2pic.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
    assert set(o2pic.EXPORTS) <= set(names)


def test_null_handle_calls_fail_cleanly(lib):
    # argument checks that need no GPU: a NULL handle is PIC_EINVAL
    assert lib.pic_step(None, 1) == 1
    assert lib.pic_set_launch(None, 0, 1) == 1
    assert lib.pic_get_launch(None, 0, None, None) == 1
    assert lib.pic_kernel_timing(None, 0, None, None, None, 0) == 1
    assert lib.pic_last_error(None)


def test_workspace_size_and_validation(lib):
    d = inputs.cfg1()
    n = o2pic.workspace_size([d], inputs.xs_tables())
    # particle pools dominate: two buffers x (int32 cell + 4 FP64 values) per slot
    slots = sum(int(np.ceil(c / 1024.0)) * 1024 for c in d.capacity)
    assert n >= 2 * slots * (4 + 4 * 8)
    assert o2pic.workspace_size([d], inputs.xs_tables(), fp64=False) < n
    bad = inputs.cfg1(n_cells=1)
    with pytest.raises(o2pic.PicError):
        o2pic.workspace_size([bad], inputs.xs_tables())
    # gas channels of one projectile must share one grid
    t = inputs.xs_tables()
    t[1] = dict(t[1], E_eV=t[1]["E_eV"] * 1.01)
    with pytest.raises(o2pic.PicError, match="share one grid"):
        o2pic.workspace_size([d], t)
    # mixed precision across discharges is rejected
    with pytest.raises(o2pic.PicError):
        o2pic.workspace_size([inputs.cfg1(), inputs.cfg1(fp64=False)], inputs.xs_tables())


def test_batched_workspace_grows_with_discharges(lib):
    one = o2pic.workspace_size([inputs.cfg1(n_op=1000)], inputs.xs_tables())
    two = o2pic.workspace_size([inputs.cfg1(n_op=1000), inputs.cfg1(n_op=1000, n_cells=64)],
                               inputs.xs_tables())
    assert two > one


def _c_layout(tmp_path, struct, fields, header="o2pic.h", incdir=os.path.join(ROOT, "include")):
    """offsetof of each field and sizeof, as the C compiler lays out the
    struct declared in the header"""
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', f'#include "{header}"', "int main(void) {"]
    for f in fields:
        lines.append(f'    printf("%zu\\n", offsetof({struct}, {f}));')
    lines += [f'    printf("%zu\\n", sizeof({struct}));', "    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", incdir, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("cls", [o2pic.pic_config, o2pic.pic_xs_table])
def test_binding_struct_layout_matches_the_header(tmp_path, cls):
    names = [f[0] for f in cls._fields_]
    c = _c_layout(tmp_path, cls.__name__, names)
    py = [getattr(cls, n).offset for n in names] + [C.sizeof(cls)]
    assert c == py, list(zip(names + ["sizeof"], c, py))


def test_oracle_binding_config_layout_matches_its_header(tmp_path):
    import oracle
    cls = oracle._Cfg
    names = [f[0] for f in cls._fields_]
    c = _c_layout(tmp_path, "orc_cfg", names, "o2pic_oracle.h", os.path.join(ROOT, "oracle"))
    py = [getattr(cls, n).offset for n in names] + [C.sizeof(cls)]
    assert c == py, list(zip(names + ["sizeof"], c, py))


def test_kernel_kinds_of_the_binding_match_the_header():
    src = open(os.path.join(ROOT, "include", "o2pic.h")).read()
    kinds = dict((k.lower(), int(v)) for k, v in re.findall(r"PIC_KERNEL_([A-Z_]+)\s*=\s*(\d+)", src))
    assert kinds == o2pic.KERNELS
