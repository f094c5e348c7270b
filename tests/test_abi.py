"""The C ABI library loads and exports every entry point that include/akra.h declares, and
argument errors come back as statuses (these run without a GPU: validation happens before
any CUDA call)."""
import os
import re

import pytest

from paper_2606_06175_gb300 import akra as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "akra.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(akra_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_06175_gb300 import build

    build.build()
    return A.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(A.EXPORTS)


def test_version(lib):
    assert "sm_103a" in A.akra_version()


@pytest.mark.parametrize("nside,lmax", [(0, 10), (4096, 100), (16, 1), (16, 65), (-3, 4)])
def test_plan_create_rejects_bad_sizes(lib, nside, lmax):
    with pytest.raises(A.AkraError) as ei:
        A.akra_plan_create(nside, lmax)
    assert ei.value.status == 1
    assert "akra_plan_create" in str(ei.value)


def test_null_arguments_are_rejected(lib):
    import ctypes

    assert lib.akra_plan_create(8, 8, None) == 1
    assert lib.akra_synth_spin2(None, 0, None, None, 1, None) == 1
    assert lib.akra_apply_H(None, 0, None, None, 1, None) == 1
    assert lib.akra_cg_solve(None, 0, None, None, 1, 1e-6, 10, None, None) == 1
    assert lib.akra_set_timeout(ctypes.c_double(-1.0)) == 1
    lib.akra_set_mixed_policy.argtypes = [ctypes.c_double, ctypes.c_double]
    assert lib.akra_set_mixed_policy(-1.0, 0.5) == 1
    assert lib.akra_set_mixed_policy(0.0, 0.0) == 1
    assert lib.akra_set_mixed_policy(0.0, 2.0) == 1
    assert lib.akra_set_mixed_policy(0.0, 0.5) == 0     # the defaults
    assert lib.akra_plan_get_shape(None, 0, 1, None, None, None) == 1
    assert lib.akra_plan_set_shape(None, 0, 1, 1, 1, 1) == 1
    assert lib.akra_plan_describe(None, None) == 1
    lib.akra_plan_destroy(None)   # no-op
    assert b"NULL" in lib.akra_last_error() or len(lib.akra_last_error()) > 0


def test_set_timeout_rejects_non_finite_and_huge_budgets(lib):
    """The budget becomes a microsecond count: NaN, +inf and values beyond 1e9 s would overflow
    that conversion, so they are rejected, as are values <= 0."""
    import ctypes

    lib.akra_set_timeout.argtypes = [ctypes.c_double]
    for v in (float("inf"), float("nan"), 1e300, 1.0000001e9, 0.0, -1.0, float("-inf")):
        assert lib.akra_set_timeout(v) == 1, v
    assert lib.akra_set_timeout(1e9) == 0
    assert lib.akra_set_timeout(3600.0) == 0     # back to the default
