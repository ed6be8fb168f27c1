"""The C-ABI library loads and exports every entry point include/muca.h declares
(no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "muca.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(muca_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_1212_3975_gb300 import build
    return build.build()


def test_header_parses():
    names = header_functions()
    assert "muca_init" in names and "muca_reweight" in names and len(names) >= 20


def test_every_declared_symbol_is_exported(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(muca_\w+)", out))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_header(built):
    import paper_1212_3975_gb300 as m
    lib = m.lib()
    for name in header_functions():
        assert hasattr(lib, name)
    assert set(header_functions()) == set(m.declared_symbols())


def test_errors_without_device_or_bad_args(built):
    import paper_1212_3975_gb300 as m
    # argument errors are reported before any device work
    for args in ((0, 7, 2, 8, 1), (0, 8, 3, 8, 1), (1, 32, 3, 8, 1), (0, 8, 2, 0, 1),
                 (2, 8, 2, 8, 1), (0, 8, 2, 8, 1 << 62)):
        with pytest.raises(m.MucaError) as ei:
            m.Muca(*args)
        assert ei.value.code == -1
