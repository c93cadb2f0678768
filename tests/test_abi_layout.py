"""The ctypes mirrors of include/tgp.h's structs have the C layout: the size
of every struct and the offset of every field, as the C compiler lays them
out (a small program built against the header with the host's gcc)."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2103_07512_gb300 as tgp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIRRORS = {
    "tgp_config": tgp.Config, "tgp_stats": tgp.Stats, "tgp_target_tokens": tgp.TargetTokens,
    "tgp_server_config": tgp.ServerConfig, "tgp_job": tgp.Job, "tgp_job_info": tgp.JobInfo,
    "tgp_server_stats": tgp.ServerStats, "tgp_evolve_config": tgp.EvolveConfig,
}


def test_struct_sizes_and_field_offsets_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tgp.h"', "int main(void) {"]
    for cname, cls in MIRRORS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            name, field, value = line.split()
            c[(name, field)] = int(value)
    for cname, cls in MIRRORS.items():
        assert c[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert c[(cname, field)] == getattr(cls, field).offset, f"{cname}.{field}"
