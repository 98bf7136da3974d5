"""Failure detection on the host (CPU, no GPU work): the serving admission
refuses what cannot run instead of failing later on the device.

* A request whose footprint estimate exceeds the whole HBM budget is refused
  at submission (an allocation failure made on the host).
* A request with a negative slab count is refused at submission too.
"""
import pytest

stfem = pytest.importorskip("paper_2303_06742_gb300")


def test_admission_refuses_oversized_and_device_less_requests():
    prob = stfem.Problem(2, 8, 3, 2, 1, 0.01, problem=stfem.PROBLEM_SIN)
    need = stfem.estimate_bytes(prob, stfem.MIXED)
    small = stfem.Server(need // 2, 1)
    try:
        with pytest.raises(stfem.StfemError) as e:
            small.submit(prob, 2)
        assert e.value.code == stfem.ERR_ARG
    finally:
        small.close()
    big = stfem.Server(1 << 40, 1)
    try:
        with pytest.raises(stfem.StfemError):
            big.submit(prob, -1)
    finally:
        big.close()
