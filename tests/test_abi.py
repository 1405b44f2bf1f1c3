"""The C-ABI library loads and exports every entry point include/corr2d.h declares.

CPU only: no compute call is made (there may be no GPU); the library is built
here with nvcc if it is missing."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "corr2d.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(corr2d_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("corr2d_create", "corr2d_destroy", "corr2d_preprocess", "corr2d_compute",
                     "corr2d_batch", "corr2d_last_error", "corr2d_synchronize"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1808_00685_gb300 as pkg
    path = pkg.build()
    lib = pkg.load(path)
    names = declared_functions()
    assert set(names) == set(pkg.EXPORTED_SYMBOLS)
    for name in names:
        assert hasattr(lib, name), f"{name} not exported"
    assert pkg.corr2d_version().startswith("corr2d-gb300")


def test_params_default_and_create_without_gpu():
    import torch
    import paper_1808_00685_gb300 as pkg
    pkg.load(pkg.build())
    p = pkg.corr2d_params_default()
    assert p.ref_mode == pkg.REF_MEAN and p.precision == pkg.PREC_SPLIT and p.norm == 0.0
    if not torch.cuda.is_available():
        with pytest.raises(pkg.Corr2dError) as ei:
            pkg.corr2d_create(0, None)
        assert ei.value.status in (pkg.ECUDA, pkg.EINVAL)
        assert pkg.corr2d_last_error(None)


def test_package_refuses_to_run_without_the_library(tmp_path):
    import paper_1808_00685_gb300 as pkg
    saved = pkg._lib
    pkg._lib = None
    try:
        with pytest.raises(RuntimeError):
            pkg.load(str(tmp_path / "missing.so"))
    finally:
        pkg._lib = saved
