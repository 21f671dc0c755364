"""The C ABI library loads and exports every entry point include/bpmf.h declares.

These run without a GPU: the library is built with nvcc for sm_103a and loaded
with ctypes; only calls that fail argument checks before touching the device
are made.
"""
import ctypes as C
import os
import re
import subprocess
from pathlib import Path

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bpmf.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"BPMF_API\s+[\w\s\*]*?\b(bpmf_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    import paper_1705_04159_gb300 as bp
    return bp.build()


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("bpmf_init", "bpmf_sample_hyper", "bpmf_sweep", "bpmf_step", "bpmf_predict",
                 "bpmf_get_state", "bpmf_set_state", "bpmf_destroy", "bpmf_strerror"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s+(\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    # nothing but the ABI is exported
    extra = [n for n in exported if n.startswith("bpmf") and n not in _declared()]
    assert not extra
    lib = C.CDLL(libpath)
    for n in _declared():
        assert hasattr(lib, n)


def test_python_binding_names_match_abi(libpath):
    import paper_1705_04159_gb300 as bp
    for n in _declared():
        if n in ("bpmf_last_error",):
            continue
        assert hasattr(bp, n), n


def test_status_strings_and_defaults(libpath):
    import paper_1705_04159_gb300 as bp
    assert bp.bpmf_strerror(0) == "ok"
    assert "invalid" in bp.bpmf_strerror(-1)
    cfg = bp.bpmf_config_default(16)
    assert cfg.K == 16 and cfg.nu0 == 16.0 and cfg.path == bp.PATH_MIXED
    assert cfg.light_max == -1 and cfg.hub_min == -1 and cfg.tiny_max == -1
    assert cfg.autotune == 0



@pytest.mark.parametrize("K", [0, 129])
def test_init_rejects_bad_K_before_touching_the_device(libpath, K):
    import numpy as np
    import paper_1705_04159_gb300 as bp
    cfg = bp.bpmf_config_default(max(K, 1))
    cfg.K = K
    with pytest.raises(bp.BpmfError) as e:
        bp.bpmf_init(4, 4, np.zeros(1, np.int32), np.zeros(1, np.int32), np.ones(1, np.float32),
                     cfg, stream=0)
    assert e.value.code == bp.EINVAL


def test_init_rejects_bad_prior(libpath):
    import numpy as np
    import paper_1705_04159_gb300 as bp
    cfg = bp.bpmf_config_default(4)
    cfg.nu0 = 2.0  # must exceed K - 1
    with pytest.raises(bp.BpmfError) as e:
        bp.bpmf_init(4, 4, np.zeros(1, np.int32), np.zeros(1, np.int32), np.ones(1, np.float32),
                     cfg, stream=0)
    assert e.value.code == bp.EINVAL


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1705_04159_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "bpmf_oracle" not in txt, f


@pytest.mark.parametrize("pyname,ctype", [("Config", "bpmf_config"), ("Job", "bpmf_job"),
                                           ("JobResult", "bpmf_job_result")])
def test_struct_mirrors_match_the_c_layout(tmp_path, pyname, ctype):
    """The ctypes mirrors have the size and field offsets gcc gives the C structs."""
    import shutil
    import paper_1705_04159_gb300 as bp
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    cls = getattr(bp, pyname)
    names = [f[0] for f in cls._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({ctype}, {n}));\n' for n in names)
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"bpmf.h\"\n"
                   f"int main(void) {{\n  printf(\"%zu\\n\", sizeof({ctype}));\n" + body +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    root = Path(__file__).resolve().parents[1]
    subprocess.run(["gcc", "-I", str(root / "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got[0] == C.sizeof(cls)
    assert got[1:] == [getattr(cls, n).offset for n in names]


@pytest.mark.parametrize("name,args", [
    ("bpmf_sample_hyper", (0,)), ("bpmf_sweep", (1,)), ("bpmf_step", ()),
    ("bpmf_set_graph", (1,)), ("bpmf_test_rmse", (None, None)),
    ("bpmf_get_state", (None, None, None, None, 0)), ("bpmf_get_thresholds", (0, None)),
    ("bpmf_get_sweep_info", (0, None, None)), ("bpmf_set_timing", (1,)),
    ("bpmf_set_limits", (64, 0)), ("bpmf_set_test_hold", (1,)),
])
def test_null_handle_is_rejected_with_a_message(libpath, name, args):
    """Every entry point that takes a handle checks it before anything else
    and says which call rejected its arguments."""
    import paper_1705_04159_gb300 as bp
    L = bp.lib()
    assert getattr(L, name)(None, *args) == bp.EINVAL
    assert L.bpmf_last_error().decode().startswith(name + ": invalid argument")


def test_missing_library_fails_loudly():
    """Without the built CUDA library every call raises: there is no CPU or
    eager fallback behind the binding."""
    code = (
        "import numpy as np\n"
        "import paper_1705_04159_gb300 as bp\n"
        "bp._build.LIB = '/nonexistent/libbpmf_missing.so'\n"
        "try:\n"
        "    bp.Sampler(4, 4, np.zeros(1, np.int32), np.zeros(1, np.int32),\n"
        "               np.ones(1, np.float32), K=2)\n"
        "except RuntimeError as e:\n"
        "    assert 'is not built' in str(e), e\n"
        "    print('raised')\n"
    )
    import sys
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == "raised"


@pytest.mark.parametrize("field,value", [
    ("alpha", 0.0), ("alpha", -1.0), ("alpha", float("nan")), ("alpha", float("inf")),
    ("beta0", float("inf")), ("beta0", 0.0), ("nu0", float("nan")), ("nu0", float("inf")),
    ("pivot_rel", 1.0), ("pivot_rel", -0.1), ("pivot_rel", float("nan")), ("tiny_max", 33),
])
def test_init_rejects_non_positive_or_non_finite_settings(libpath, field, value):
    """The row precision Lambda_s + alpha sum v v^T is positive definite for
    any alpha > 0, so the FP64 redo can only fail by rounding once alpha is
    positive and finite; the configuration is refused before the device is
    touched otherwise."""
    import numpy as np
    import paper_1705_04159_gb300 as bp
    cfg = bp.bpmf_config_default(4)
    setattr(cfg, field, value)
    with pytest.raises(bp.BpmfError) as e:
        bp.bpmf_init(4, 4, np.zeros(1, np.int32), np.zeros(1, np.int32), np.ones(1, np.float32),
                     cfg, stream=0)
    assert e.value.code == bp.EINVAL


def test_limits_reject_a_gamma_cap_above_the_default(libpath):
    import paper_1705_04159_gb300 as bp
    L = bp.lib()
    assert L.bpmf_set_limits(None, 65, 0) == bp.EINVAL
