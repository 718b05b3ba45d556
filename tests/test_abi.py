"""The C-ABI library loads and exports what include/pa.h declares (no GPU needed)."""
import os
import re

import pytest

import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "pa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_02372_gb300 import build
    build.build()
    return binding.load()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert "pa_hash" in names and "pa_hash_batched" in names and "pa_plan" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in pa.h but not exported"
        assert name in binding.SIGNATURES, f"{name} has no binding"


def test_strerror_and_version(lib):
    for code in range(0, -8, -1):
        assert pkg.pa_strerror(code) and pkg.pa_strerror(code) != "unknown status"
    assert pkg.pa_strerror(-99) == "unknown status"
    assert pkg.pa_version() >= 100


def test_plan_query_validates(lib):
    with pytest.raises(pkg.PAError) as e:
        pkg.pa_plan_query(0, 5)
    assert e.value.status == binding.PA_ERR_INVALID
    with pytest.raises(pkg.PAError):
        pkg.pa_plan_query(5, 0)
    with pytest.raises(pkg.PAError):
        pkg.pa_plan_query(5, 5, binding.make_opts(path=17))


@pytest.mark.parametrize("n,m", [(1, 1), (100_003, 25_000), (1_000_000, 500_000)])
def test_plan_query_direct(lib, n, m):
    d = pkg.pa_plan_query(n, m, binding.make_opts(path="direct"))
    assert d["path_name"] == "direct" and d["n"] == n and d["m"] == m
    assert d["workspace_bytes"] >= 4 * ((n + 31) // 32)
