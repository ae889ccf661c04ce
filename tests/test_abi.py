"""CPU checks of the C ABI boundary: the library loads, exports every symbol
that include/qaoa.h declares, and its host-only entry points (allocation,
validation) behave as Sec. 3.1 states.  No GPU compute is called."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2606_26297_b300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def q():
    build_lib.build()
    from paper_2606_26297_b300 import qaoa
    return qaoa


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(qaoa_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(q):
    lib = ctypes.CDLL(q.LIB_PATH)
    names = _declared_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name


def test_binding_names_match_abi(q):
    for name in _declared_functions():
        assert hasattr(q, name), name


def test_partition_balanced_contiguous(q):
    """Sec. 3.1: balanced capacities floor(n/M) + [m < n mod M]; contiguous fill."""
    assert list(q.qaoa_partition(30, 3)) == [0] * 10 + [1] * 10 + [2] * 10
    assert list(q.qaoa_partition(7, 3)) == [0, 0, 0, 1, 1, 2, 2]
    assert list(q.qaoa_partition(6, 2, caps=[4, 4])) == [0, 0, 0, 0, 1, 1]


def test_partition_manual_and_validation(q):
    assert list(q.qaoa_partition(6, 2, manual=[0, 0, 1, 1, 0, 1])) == [0, 0, 1, 1, 0, 1]
    with pytest.raises(q.QaoaError) as e:          # capacity exceeded
        q.qaoa_partition(6, 2, caps=[2, 4], manual=[0, 0, 0, 1, 1, 1])
    assert e.value.status == q.QAOA_ERR_ALLOCATION
    with pytest.raises(q.QaoaError) as e:          # QPU 1 unused
        q.qaoa_partition(4, 2, manual=[0, 0, 0, 0], caps=[4, 4])
    assert e.value.status == q.QAOA_ERR_ALLOCATION
    with pytest.raises(q.QaoaError) as e:          # total capacity too small
        q.qaoa_partition(6, 2, caps=[2, 2])
    assert e.value.status == q.QAOA_ERR_ALLOCATION
    with pytest.raises(q.QaoaError) as e:
        q.qaoa_partition(3, 4)
    assert e.value.status == q.QAOA_ERR_INVALID_ARG


def test_bitstring_order(q):
    """Sec. 3.6: the logical string lists z_1..z_n; bit i of x is z_{i+1}.
    Qiskit's display string is the reverse."""
    x = 0b001101
    assert q.bitstring(x, 6) == "101100"
    assert q.bitstring(x, 6) == format(x, "06b")[::-1]


def test_ctx_create_without_gpu_fails_cleanly(q):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(q.QaoaError) as e:
        q.qaoa_ctx_create(0)
    assert e.value.status in (q.QAOA_ERR_CUDA, q.QAOA_ERR_INVALID_ARG)
    assert q.qaoa_last_error()
