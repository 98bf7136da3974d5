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


@pytest.mark.parametrize("dim,r,form", [(2, 2, 0), (2, 3, 1), (3, 2, 0)])
def test_galerkin_structure_rejects_a_dropped_entry(dim, r, form):
    """The coarse operators are node-level Galerkin products P^T A_l P: each
    node's blocks are read from the rows of its displacement component 0 and
    every other component's rows must repeat that pattern.  A level with one
    entry removed from a u- or v-equation row (component 1's first or last
    entry: a shifted pattern or a strict prefix of component 0's; or
    component 0's own last entry) is rejected with ERR_STATE, instead of
    giving a coarse operator that is no longer P^T A_l P."""
    n = 4
    prob = stfem.Problem(dim, n, 2, r, 1, 0.01, problem=stfem.PROBLEM_SIN, form=form)
    stfem.host_galerkin_check(prob, level=1)  # the level as assembled passes
    R = dim * (r * n + 1) ** dim  # u-equation rows: d per Q_r node
    for row, last in [(1, True), (1, False), (0, True), (R + 1, True), (R + 1, False)]:
        with pytest.raises(stfem.StfemError) as e:
            stfem.host_galerkin_check(prob, level=1, drop_row=row, drop_last=last)
        assert e.value.code == stfem.ERR_STATE, (row, last)
        assert "node-block structure" in str(e.value)
    with pytest.raises(stfem.StfemError) as e:
        stfem.host_galerkin_check(prob, level=0)
    assert e.value.code == stfem.ERR_ARG
