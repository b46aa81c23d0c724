"""Layout of the built objects (CPU only; needs the in-tree build).

The line-decomposed operator kernels read their even-odd coefficients from
`__constant__` arrays that every translation unit owns a copy of and fills
itself (no relocatable device code).  That is only consistent if each
per-order, per-precision operator launcher -- and with it every kernel it
launches -- is compiled in exactly one object, the one named for that order
and precision; a second, implicit instantiation elsewhere would let the linker
pair a launcher with another unit's kernels and constants."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(os.path.dirname(HERE), "paper_2506_09435_gb300", "_build")


def defined(obj):
    out = subprocess.run(["nm", "-C", "--defined-only", obj], capture_output=True, text=True, check=True).stdout
    return out.splitlines()


@pytest.mark.skipif(not os.path.isdir(BUILD) or shutil.which("nm") is None, reason="needs the in-tree build and nm")
def test_each_operator_instantiation_lives_in_its_own_object():
    objs = sorted(f for f in os.listdir(BUILD) if f.endswith(".o"))
    if not any(f.startswith("ax_n") for f in objs):
        pytest.skip("library not built")
    where = {}
    pat = re.compile(r"fnpf::launch_ax_n<(double|float), (\d)>\(")
    for f in objs:
        for line in defined(os.path.join(BUILD, f)):
            m = pat.search(line)
            if m:
                where.setdefault((m.group(1), int(m.group(2))), []).append(f)
    expected = {(t, n) for t in ("double", "float") for n in range(2, 10)}
    assert set(where) == expected, sorted(set(where) ^ expected)
    for (t, n), files in where.items():
        want = "ax_n%d_%s.o" % (n, "f64" if t == "double" else "f32")
        assert files == [want], ((t, n), files)
