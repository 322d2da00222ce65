"""The C-ABI library loads and exports every symbol include/hhg.h declares (no GPU needed)."""

import pytest

from paper_1908_08666_gb300 import binding as B


def test_library_exports_declared_symbols():
    lib = B.load()
    declared = B.declared_symbols()
    assert len(declared) >= 10
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    # every declared entry point has a Python wrapper of the same name
    assert not [s for s in declared if not hasattr(B, s)]


def test_create_without_gpu_fails_loudly():
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(B.HhgError):
        B.hhg_create(0, 0)
