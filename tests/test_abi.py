"""Host-side checks of the C-ABI library (no GPU needed): it builds for sm_103a, loads, exports
every entry point that include/tof.h declares, rejects use without a device, and the product
package never reaches into the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tof.h")).read()
    return re.findall(r"^\s*(?:tof_status|const char\*|uint64_t)\s+(tof_\w+)\(", src, re.M)


def test_header_and_binding_agree():
    from paper_2605_11536_gb300 import tof
    assert sorted(_declared()) == sorted(tof.EXPORTS)
    assert len(tof.EXPORTS) == 30


def test_library_builds_and_exports_every_symbol():
    from paper_2605_11536_gb300 import tof
    L = tof.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2605_11536_gb300 import tof
    with pytest.raises(tof.TofError):
        tof.tof_create(0)


def test_product_does_not_use_oracle():
    pkg = os.path.join(ROOT, "paper_2605_11536_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "tof_oracle" not in txt, f


def test_struct_sizes_match_header():
    """ctypes layouts of the binding equal the C layouts (compiled probe of include/tof.h)."""
    import ctypes as C
    import subprocess
    import tempfile
    from paper_2605_11536_gb300 import tof
    src = '#include <stdio.h>\n#include "tof.h"\nint main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(tof_material),' \
          ' sizeof(tof_sensor), sizeof(tof_emitter), sizeof(tof_gate), sizeof(tof_bins), sizeof(tof_params), sizeof(tof_job),' \
          ' sizeof(tof_tuning));}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    assert sizes == [C.sizeof(t) for t in (tof.tof_material, tof.tof_sensor, tof.tof_emitter, tof.tof_gate,
                                             tof.tof_bins, tof.tof_params, tof.tof_job, tof.tof_tuning)]
