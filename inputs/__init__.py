"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Only data: problem sizes, coefficients and random draws.  No arithmetic of
the method lives here.  Workload shapes follow the paper's setting (Sec. 5:
unit boxes, uniform refinement, Taylor-Hood pairs, dG(k) slabs) at the
sizes of the benchmarked configurations.
"""
import numpy as np

SEED = 20230312


def lame_from_young(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def case(name, seed=SEED):
    """Keyword arguments of a problem instance (for paper_2303_06742_gb300.Problem
    and for the oracle's Instance), by name."""
    rng = np.random.default_rng(seed)
    if name == "c1_2d_q2_k1_8":  # 2D unit square 8x8, Q2/Q1, k=1, 3 levels
        return dict(dim=2, n=8, levels=3, r=2, k=1, tau=0.01, slabs=10, rho=1.0, alpha=1.0, c0=1.0,
                    lam=1.0, mu=1.0, kappa=1.0, problem="sin", tol=1e-10)
    if name == "c1_2d_q2_k1_32":  # the 8x8 recipe on 32x32, 4 levels (1,089 fine patches)
        return dict(dim=2, n=32, levels=4, r=2, k=1, tau=0.01, slabs=2, rho=1.0, alpha=1.0, c0=1.0,
                    lam=1.0, mu=1.0, kappa=1.0, problem="sin", tol=1e-10)
    if name == "bd_2d_q2_k1_8":  # nonzero boundary data: Dirichlet and Neumann faces, random cells
        return dict(dim=2, n=8, levels=3, r=2, k=1, tau=0.01, slabs=2, rho=1.0, alpha=0.9, c0=0.5,
                    lo=[0.0, -0.25], hi=[1.0, 1.25], lam_cell=np.exp(rng.uniform(0.0, 1.5, 64)),
                    mu_cell=np.exp(rng.uniform(-0.5, 0.5, 64)), kappa_cell=np.exp(rng.standard_normal(64)),
                    bc_u=[0, 1, 0, 0], bc_p=[1, 0, 0, 0], problem="trace", tol=1e-10)
    if name == "bd_2d_q3_k2_8":
        return dict(dim=2, n=8, levels=3, r=3, k=2, tau=1e-3, slabs=2, rho=1.0, alpha=1.0, c0=1e-2,
                    lam=3.0, mu=1.5, kappa_cell=np.exp(rng.standard_normal(64)),
                    bc_u=[0, 0, 1, 0], bc_p=[0, 1, 0, 0], problem="trace", tol=1e-10)
    if name == "bd_3d_q2_k1_4":
        return dict(dim=3, n=4, levels=2, r=2, k=1, tau=1e-2, slabs=2, rho=1.0, alpha=0.5, c0=1.0,
                    lam=2.0, mu=1.0, kappa=0.1, bc_u=[0, 1, 0, 0, 0, 1], bc_p=[1, 0, 0, 0, 0, 0],
                    problem="trace", tol=1e-10)
    if name == "bd_sin_neumann_2d_q2_k1_8":  # zero traces, Neumann data of the exact solution
        return dict(dim=2, n=8, levels=3, r=2, k=1, tau=0.01, slabs=2, rho=1.0, alpha=1.0, c0=1.0,
                    lam=1.0, mu=1.0, kappa=1.0, bc_u=[1, 0, 0, 1], bc_p=[0, 0, 1, 0], problem="sin", tol=1e-10)
    if name in ("aniso_2d_q3_k2_8", "aniso_bd_2d_q2_k1_8", "aniso_3d_q2_k1_4"):
        # a symmetric positive definite permeability tensor per cell, with
        # off-diagonal entries as large as the diagonal ones (K = A A^T + 0.3 I)
        dim = 3 if name.startswith("aniso_3d") else 2
        n = 4 if dim == 3 else 8
        A = rng.standard_normal((n ** dim, dim, dim))
        K = np.einsum("cij,ckj->cik", A, A) + 0.3 * np.eye(dim)[None]
        if name == "aniso_2d_q3_k2_8":
            return dict(dim=2, n=8, levels=3, r=3, k=2, tau=1e-3, slabs=2, rho=1.0, alpha=1.0, c0=1e-2,
                        lam=3.0, mu=1.5, K_cell=K, problem="sin", tol=1e-10)
        if name == "aniso_bd_2d_q2_k1_8":
            return dict(dim=2, n=8, levels=3, r=2, k=1, tau=0.01, slabs=2, rho=1.0, alpha=0.9, c0=0.5,
                        lam=2.0, mu=1.0, K_cell=K, bc_u=[0, 1, 0, 0], bc_p=[1, 0, 0, 1], problem="trace",
                        tol=1e-10)
        return dict(dim=3, n=4, levels=2, r=2, k=1, tau=1e-2, slabs=2, rho=1.0, alpha=0.5, c0=1.0,
                    lam=2.0, mu=1.0, K_cell=K, bc_u=[0, 0, 0, 1, 0, 0], bc_p=[0, 0, 0, 0, 1, 0],
                    problem="trace", tol=1e-10)
    if name == "c2_2d_q3_k2_64":  # 2D 64x64, 5 levels, Q3/Q2, k=2, random materials
        lam = float(np.exp(rng.uniform(np.log(0.5), np.log(50.0))))
        mu = float(np.exp(rng.uniform(np.log(0.5), np.log(50.0))))
        kap = np.exp(rng.standard_normal(64 * 64))
        return dict(dim=2, n=64, levels=5, r=3, k=2, tau=1e-3, slabs=20, rho=1.0, alpha=1.0, c0=1e-2,
                    lam=lam, mu=mu, kappa_cell=kap, problem="sin", tol=1e-8)
    if name == "c2_small_2d_q3_k2_8":  # same recipe, 8x8 / 3 levels (oracle-sized)
        lam = float(np.exp(rng.uniform(np.log(0.5), np.log(50.0))))
        mu = float(np.exp(rng.uniform(np.log(0.5), np.log(50.0))))
        kap = np.exp(rng.standard_normal(8 * 8))
        return dict(dim=2, n=8, levels=3, r=3, k=2, tau=1e-3, slabs=3, rho=1.0, alpha=1.0, c0=1e-2,
                    lam=lam, mu=mu, kappa_cell=kap, problem="sin", tol=1e-8)
    if name == "c3_small_3d_q2_k1_4":  # thermoelastic set, 3D 4^3, 2 levels
        return dict(dim=3, n=4, levels=2, r=2, k=1, tau=1e-2, slabs=2, rho=1.0, alpha=0.5, c0=1.0,
                    lam=2.0, mu=1.0, kappa=0.1, problem="sin", tol=1e-8)
    if name == "c3_3d_q2_k1_16":
        return dict(dim=3, n=16, levels=4, r=2, k=1, tau=1e-2, slabs=10, rho=1.0, alpha=0.5, c0=1.0,
                    lam=2.0, mu=1.0, kappa=0.1, problem="sin", tol=1e-8)
    if name == "c5_small_3d_pulse":  # layered box [0,2]^2 x [0,1], 4x4x2 cells
        n = (4, 4, 2)
        kap, mu = layered(n, 1.0)
        return dict(dim=3, n=n, levels=2, r=2, k=1, tau=5e-3, slabs=2, lo=[0, 0, 0], hi=[2, 2, 1],
                    rho=1.0, alpha=1.0, c0=1.0, lam=1.0, mu_cell=mu, kappa_cell=kap, problem="pulse",
                    bc_u=[1, 1, 1, 1, 0, 1], bc_p=[1, 1, 1, 1, 1, 0], tol=1e-8)
    if name == "c5_3d_pulse_32":  # layered box [0,2]^2 x [0,1], 32^3 cells, 4 levels
        n = (32, 32, 32)
        kap, mu = layered(n, 1.0)
        return dict(dim=3, n=n, levels=4, r=2, k=1, tau=5e-3, slabs=40, lo=[0, 0, 0], hi=[2, 2, 1],
                    rho=1.0, alpha=1.0, c0=1.0, lam=1.0, mu_cell=mu, kappa_cell=kap, problem="pulse",
                    bc_u=[1, 1, 1, 1, 0, 1], bc_p=[1, 1, 1, 1, 1, 0], tol=1e-8)
    raise KeyError(name)


def served_with_pulse(n_small=16):
    """The layered 32^3 pulse march (40 slabs) submitted together with
    n_small 3D 16^3 thermoelastic marches (10 slabs each, data phases
    t0 = 0.05 i), all at time 0."""
    out = [dict(case("c5_3d_pulse_32"), arrival=0.0)]
    for i in range(n_small):
        out.append(dict(case("c3_3d_q2_k1_16"), t0=0.05 * i, arrival=0.0))
    return out


def layered(n, top_z_split):
    """Two horizontal layers split at z = 0.5: lower kappa = 1, mu = 1; upper
    kappa = 1e-3, mu = 10 (per cell, cells lexicographic with x fastest)."""
    nx, ny, nz = n
    kap = np.empty(nx * ny * nz)
    mu = np.empty(nx * ny * nz)
    for z in range(nz):
        upper = (z + 0.5) / nz * top_z_split > 0.5
        sl = slice(z * nx * ny, (z + 1) * nx * ny)
        kap[sl] = 1e-3 if upper else 1.0
        mu[sl] = 10.0 if upper else 1.0
    return kap, mu


def serving_stream(n_requests=256, seed=SEED, mean_gap_s=2e-3, meshes=(16, 32, 64, 128),
                   degrees=((2, 1), (3, 2)), slabs=(5, 50)):
    """Request stream of the serving workload: Poisson arrivals (exponential
    gaps, mean 2 ms), square 2D meshes drawn uniformly from `meshes` (GMG down
    to 4x4), (r, k) uniformly from `degrees`, the slab count uniform in
    `slabs`, materials drawn as for the 64x64 workload (lambda, mu
    log-uniform in [0.5, 50] per request, kappa lognormal per cell,
    c0 = 1e-2, tau = 1e-3), the sine manufactured solution, tol 1e-8."""
    rng = np.random.default_rng(seed + 4)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += float(rng.exponential(mean_gap_s))
        n = int(rng.choice(meshes))
        r, k = degrees[int(rng.integers(len(degrees)))]
        levels = int(round(np.log2(n / 4))) + 1
        lam = float(np.exp(rng.uniform(np.log(0.5), np.log(50.0))))
        mu = float(np.exp(rng.uniform(np.log(0.5), np.log(50.0))))
        kap = np.exp(rng.standard_normal(n * n))
        out.append(dict(arrival=t, dim=2, n=n, levels=levels, r=r, k=k, tau=1e-3,
                        slabs=int(rng.integers(slabs[0], slabs[1] + 1)), rho=1.0, alpha=1.0, c0=1e-2,
                        lam=lam, mu=mu, kappa_cell=kap, problem="sin", tol=1e-8))
    return out
