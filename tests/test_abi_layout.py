"""The ctypes mirrors of the C structs in include/dr.h have the C layout:
every field at the same offset and every struct the same size, as a C
compiler sees the header (gcc, no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2201_13309_gb300 import dr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "dr_geometry": dr.Geometry,
    "dr_plan_options": dr.PlanOptions,
    "dr_plan_info": dr.PlanInfo,
    "dr_job": dr.Job,
    "dr_batch_options": dr.BatchOptions,
    "dr_batch_info": dr.BatchInfo,
    "dr_server_options": dr.ServerOptions,
    "dr_request_times": dr.RequestTimes,
    "dr_server_stats": dr.ServerStats,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include "dr.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("%s size %zu\\n", "{cname}", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("%s %s %zu\\n", "{cname}", "{field}", '
                         f"offsetof({cname}, {field}));")
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        layout[(cname, field)] = int(value)
    return layout


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    cls = STRUCTS[cname]
    assert ctypes.sizeof(cls) == c_layout[(cname, "size")], cname
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(cname, field)], (cname, field)
