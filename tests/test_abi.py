"""The C-ABI library loads and exports every entry point include/icm.h declares;
argument validation that needs no GPU rejects bad input with ICM_EINVAL."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "icm.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(icm_[a-z_0-9]+)\s*\(", text)) - {"icm_alloc_fn", "icm_free_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_1212_6427_gb300 import build
    build.build_library()
    import paper_1212_6427_gb300 as icm
    return icm


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("icm_create", "icm_add_blobs", "icm_step", "icm_read_state", "icm_write_state",
                     "icm_destroy", "icm_last_error", "icm_set_blob_forces"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = ctypes.CDLL(lib.binding.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert missing == []
    # and the binding wraps each of them under the same name
    assert set(_declared()) <= set(lib.binding.SIGNATURES)
    for n in _declared():
        assert hasattr(lib.binding, n) or n == "icm_set_default_allocator"


@pytest.mark.parametrize("bad", [
    dict(grid=(32, 32, 7)),            # not 2^a 3^b
    dict(grid=(32, 32, 6)),            # smaller than 2 * kernel width
    dict(grid=(32, 1024, 32)),         # too large
    dict(kernel=5),
    dict(h=0.0), dict(rho=-1.0), dict(eta=0.0), dict(dt=0.0), dict(kT=-1e-3),
    dict(h=float("nan")),
    dict(precision=16),
    dict(flags=0x6),                   # two slip options
    dict(flags=0x100),
])
def test_create_rejects_invalid_arguments(lib, bad):
    args = dict(grid=(32, 32, 32), h=1.0, rho=1.0, eta=1.0, kT=1e-3, dt=0.05, kernel=4, seed=1, precision=32,
                flags=0)
    args.update(bad)
    with pytest.raises(lib.IcmError) as ei:
        lib.icm_create(args["grid"], args["h"], args["rho"], args["eta"], args["kT"], args["dt"], args["kernel"],
                       args["seed"], args["precision"], args["flags"], None)
    assert ei.value.status == lib.ICM_EINVAL
    assert lib.icm_last_error()


def test_philox_rejects_negative_count(lib):
    with pytest.raises(lib.IcmError):
        lib.icm_op_philox(-1, (0, 0, 0, 0), (0, 0))


def test_kernel_volume_host_arithmetic(lib):
    """dV = h^3 / (sum phi^2)^3: the paper's 8 h^3 for the 3-point kernel and (8/3)^3 h^3
    for the 4-point kernel (host arithmetic, no GPU)."""
    assert lib.icm_kernel_volume(3, 1.0) == 8.0
    assert abs(lib.icm_kernel_volume(3, 0.5) - 1.0) < 1e-15
    assert abs(lib.icm_kernel_volume(4, 1.0) - 512.0 / 27.0) < 1e-13
    for kernel, h in ((5, 1.0), (3, 0.0), (4, float("inf"))):
        with pytest.raises(lib.IcmError) as ei:
            lib.icm_kernel_volume(kernel, h)
        assert ei.value.status == lib.ICM_EINVAL
