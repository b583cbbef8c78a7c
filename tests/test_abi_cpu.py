"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point that include/bfvm.h declares, and rejects bad
arguments on the host with the documented status codes."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bf():
    from paper_2110_13368_gb300 import build, bfvm
    build.build()
    bfvm.load_library()
    return bfvm


def header_functions():
    text = open(os.path.join(ROOT, "include", "bfvm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bfvm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(bf):
    lib = bf.load_library()
    names = header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(bf.EXPORTED) == names


def test_status_strings(bf):
    for code, name in bf.STATUS_NAMES.items():
        assert bf.bfvm_status_string(code) == name


@pytest.mark.parametrize("kw,msg", [
    (dict(nx=0), "grid edges"),
    (dict(nz=-3), "grid edges"),
    (dict(dx=0.0), "dx"),
    (dict(dx=math.inf), "dx"),
    (dict(dt=-1.0), "dt"),
    (dict(precision=16), "precision"),
    (dict(D=[-1.0]), "D must"),
    (dict(lam=[math.nan]), "lambda"),
    (dict(bc_kind=[2]), "bc_kind"),
    (dict(bc_value=[math.inf]), "bc_value"),
])
def test_create_rejects_bad_arguments_on_host(bf, kw, msg):
    args = dict(nx=4, ny=4, nz=4, dx=20.0, dt=0.01, D=[1e5], lam=[0.1], bc_kind=[0],
                bc_value=[0.0], precision=64)
    args.update(kw)
    with pytest.raises(bf.BfvmError) as ei:
        bf.bfvm_create(args["nx"], args["ny"], args["nz"], args["dx"], args["dt"], args["D"],
                       args["lam"], args["bc_kind"], args["bc_value"], args["precision"])
    assert ei.value.status == 1
    assert msg in str(ei.value)


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    from paper_2110_13368_gb300 import bfvm
    saved = bfvm._lib
    try:
        bfvm._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            bfvm.load_library(str(tmp_path / "missing.so"))
    finally:
        bfvm._lib = saved


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2110_13368_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.c" not in text, f


def test_option_keys_agree_between_header_code_and_binding():
    """Every option key the library handles is documented in include/bfvm.h
    and has a constant in the binding, and no other key is documented."""
    import re
    from paper_2110_13368_gb300 import bfvm
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    header = open(os.path.join(root, "include", "bfvm.h")).read()
    api = open(os.path.join(root, "paper_2110_13368_gb300", "csrc", "api.cu")).read()
    body = api[api.index("bfvm_set_option("):]
    body = body[:body.index("unknown option key")]
    handled = {int(k) for k in re.findall(r"case (\d+):", body)}
    documented = {int(k) for k in re.findall(r"\*\s+key (\d+)\s", header)}
    constants = {v for k, v in vars(bfvm).items() if k.startswith("OPT_")}
    assert handled == documented == constants, (handled, documented, constants)
