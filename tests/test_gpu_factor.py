"""Time-diagonal patch inverses factorised on the device (FP64 Gauss-Jordan
with partial pivoting, one CTA per patch and slot) against the host
factorisation and the oracle (needs a GPU).

Both factorisations are FP64 Gauss-Jordan with the same pivot rule, so the
inverses agree to rounding (about cond * eps); a smoothing step built on
either agrees with the other to 1e-11 and with the oracle (LAPACK inverses)
to the 1e-11 of test_gpu_parity.  In FP32 storage the two round to the same
floats except where an FP64 value sits within rounding of an FP32 midpoint:
1e-6 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _cases import case, gpu_problem, oracle_instance

CASES = ["c1_2d_q2_k1_8", "c2_small_2d_q3_k2_8", "c3_small_3d_q2_k1_4", "c5_small_3d_pulse"]


def _rel(a, b):
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-6)])
def test_device_factorisation_matches_host_and_oracle(name, precision, tol):
    import paper_2303_06742_gb300 as st
    from oracle.gmg import smooth
    c = case(name)
    O = oracle_instance(c)
    Sd = st.Solver(gpu_problem(c), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL)
    Sh = st.Solver(gpu_problem(c), precision=precision, patch_form=st.PATCH_TIME_DIAGONAL, factor_host=1)
    rng = np.random.default_rng(51)
    for l in range(1, len(O.h.levels)):
        lev = O.h.levels[l]
        b = rng.standard_normal(lev.A.shape[0])
        d0 = rng.standard_normal(lev.A.shape[0])
        dd, dh = dev(d0), dev(d0)
        Sd.smooth(l, dev(b), dd, n_sweeps=2, zero_init=False)
        Sh.smooth(l, dev(b), dh, n_sweeps=2, zero_init=False)
        ref = smooth(lev, b, d0.copy(), 0.7, 2)
        e_dh, e_do = _rel(host(dd), host(dh)), _rel(host(dd), ref)
        print(name, precision, "level", l, "device vs host", e_dh, "device vs oracle", e_do)
        assert e_dh < tol
        assert e_do < (1e-10 if precision == 0 else 1e-4)
    Sd.close()
    Sh.close()
