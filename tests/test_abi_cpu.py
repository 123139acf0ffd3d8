"""Host-side checks of the C ABI that need no GPU: the library loads, every
function declared in include/hr2.h is exported, the binding knows them, the
constants agree, and calls that touch no device behave."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1910_01070_b300 import build as B
from paper_1910_01070_b300 import hr2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header():
    with open(os.path.join(ROOT, "include", "hr2.h")) as f:
        return f.read()


def _declared_functions():
    src = re.sub(r"/\*.*?\*/", "", _header(), flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hr2.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("create_opacity_tables", "forward_model_batch", "log_likelihood_batch"):
        assert required in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in hr2.EXPORTED, name


def test_constants_match_header():
    src = _header()
    defines = dict(re.findall(r"#define\s+(HR2_\w+)\s+(-?\d+)", src))
    for name, val in defines.items():
        if hasattr(hr2, name):
            assert getattr(hr2, name) == int(val), name
    enum = dict(re.findall(r"(HR2_E\w+|HR2_OK)\s*=\s*(-?\d+)", src))
    for name, val in enum.items():
        assert getattr(hr2, name) == int(val), name


def test_host_helpers_without_device(lib):
    assert "sm_103a" in hr2.hr2_version()
    assert np.allclose(hr2.hr2_nodes_from_b(2000.0, [0.9, 0.5]), [2000.0, 1800.0, 900.0])


def test_context_creation_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hr2.Hr2Error):
        hr2.hr2_ctx_create(0, 0)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(hr2, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(hr2, "_LIB", None)
    with pytest.raises(RuntimeError):
        hr2.lib()


def _struct_fields(src, name):
    body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\}\s*" + name + ";", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            fields += re.findall(r"(\w+)\s*(?:,|$)", decl)     # "double p_top, p_bot" declares two
    return fields


@pytest.mark.parametrize("cname,pyname", [("hr2_setup_desc", "SetupDesc"), ("hr2_table_desc", "TableDesc"),
                                          ("hr2_launch_cfg", "LaunchCfg"), ("hr2_ns_state", "NsState"),
                                          ("hr2_unit_rate", "UnitRate")])
def test_binding_structs_follow_the_header(cname, pyname):
    """The ctypes mirrors list the header's fields in the header's order."""
    assert [f[0] for f in getattr(hr2, pyname)._fields_] == _struct_fields(_header(), cname)


def test_oracle_binding_struct_follows_the_c_source():
    """The oracle's ctypes model mirrors or_model field by field (test infrastructure
    has the same failure mode as the library binding)."""
    import oracle
    src = open(os.path.join(os.path.dirname(oracle.__file__), "hr2_oracle.c")).read()
    body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\}\s*or_model;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        if decl.strip():
            fields += re.findall(r"(\w+)\s*(?:,|$)", decl.strip())
    assert [f[0] for f in oracle._Model._fields_] == fields
