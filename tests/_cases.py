"""Builds the CUDA-path problem and the oracle instance from one input case."""
import numpy as np

import inputs


def _cells(c):
    n = c["n"]
    n = list(n) if hasattr(n, "__len__") else [n] * c["dim"]
    return n, int(np.prod(n))


def gpu_problem(c, hf_mode=0, form=0, pressure=0):
    import paper_2303_06742_gb300 as st
    n, nc = _cells(c)
    pid = {"sin": st.PROBLEM_SIN, "pulse": st.PROBLEM_PULSE, "none": st.PROBLEM_NONE,
           "paper_eoc": st.PROBLEM_PAPER_EOC, "paper_superconv": st.PROBLEM_PAPER_SUPERCONV,
           "trace": st.PROBLEM_TRACE}[c["problem"]]
    return st.Problem(c["dim"], n, c["levels"], c["r"], c["k"], c["tau"], lo=c.get("lo"), hi=c.get("hi"),
                      rho=c["rho"], alpha=c["alpha"], c0=c["c0"], lam=c.get("lam", 1.0), mu=c.get("mu", 1.0),
                      kappa=c.get("kappa", 1.0), lam_cell=c.get("lam_cell"), mu_cell=c.get("mu_cell"),
                      kappa_cell=c.get("kappa_cell"), bc_u=c.get("bc_u"), bc_p=c.get("bc_p"), problem=pid,
                      t0=c.get("t0", 0.0), hf_mode=hf_mode, form=form, pressure=pressure, K_cell=c.get("K_cell"))


def oracle_instance(c, omega=0.7, nsweeps=1, hf="measure", **variant):
    """``variant``: patches, averaging, absolute, form, pressure (oracle.solver.Instance)."""
    from oracle.space import Material
    from oracle.solver import Instance
    from oracle import problems as P
    n, nc = _cells(c)
    one = np.ones(nc)
    lam = c["lam_cell"] if "lam_cell" in c else c.get("lam", 1.0) * one
    mu = c["mu_cell"] if "mu_cell" in c else c.get("mu", 1.0) * one
    kap = c["kappa_cell"] if "kappa_cell" in c else c.get("kappa", 1.0) * one
    if "K_cell" in c:
        kap = np.asarray(c["K_cell"], float).reshape(nc, c["dim"], c["dim"])
    mat = Material(c["rho"], c["alpha"], c["c0"], lam, mu, kap)
    d = c["dim"]
    if c["problem"] == "sin":
        prob = P.sin_problem(d, c["rho"], c["alpha"], c["c0"])
    elif c["problem"] == "pulse":
        prob = P.PulseProblem(c["rho"], c["alpha"], c["c0"])
    elif c["problem"] == "paper_eoc":
        prob = P.paper_eoc_problem(c["rho"], c["alpha"], c["c0"])
    elif c["problem"] == "paper_superconv":
        prob = P.paper_superconv_problem(c["rho"], c["alpha"], c["c0"])
    elif c["problem"] == "trace":
        prob = P.trace_problem(d, c["rho"], c["alpha"], c["c0"])
    else:
        prob = P.zero_problem(d, c["rho"], c["alpha"], c["c0"])
    lo = c.get("lo") or [0.0] * d
    hi = c.get("hi") or [1.0] * d
    bcu = c.get("bc_u") or [0] * (2 * d)
    bcp = c.get("bc_p") or [0] * (2 * d)
    return Instance(d, lo, hi, n, c["levels"], c["r"], c["k"], mat, bcu, bcp, c["tau"], prob,
                    t0=c.get("t0", 0.0), omega=omega, nsweeps=nsweeps, hf=hf, **variant)


def case(name):
    return inputs.case(name)
