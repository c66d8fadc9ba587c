"""The ctypes mirrors of the C ABI's structs have the C layout (compiled with gcc from
include/rbd.h; no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_struct_sizes_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "include/rbd.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu\\n", sizeof(rbd_result), sizeof(rbd_profile), '
                   'sizeof(rbd_instance), sizeof(rbd_batch_result)); return 0; }\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", ROOT, str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    from paper_1503_05947_gb300 import rbd
    assert sizes == [ctypes.sizeof(rbd._Result), ctypes.sizeof(rbd._Profile), ctypes.sizeof(rbd._Instance),
                     rbd._BATCH_RESULT_BYTES]
