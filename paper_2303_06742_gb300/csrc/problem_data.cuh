// Built-in problem data: manufactured fields and sources, nodal interpolation
// or projection of the initial state, and the slab right-hand side.  Included
// by stfem.cu inside its anonymous namespace, after the device helpers.

// ---------------------------------------------------------------- problem data
__device__ void node_coord(const GeomDev &g, int deg, const int *dims, const double *ref, long idx, double *x) {
  for (int i = 0; i < 3; ++i) {
    if (i < g.dim) {
      const int a = (int)(idx % dims[i]);
      idx /= dims[i];
      const int c = min(a / deg, g.n[i] - 1);
      x[i] = g.lo[i] + g.h[i] * (c + ref[a - deg * c]);
    } else {
      x[i] = 0.0;
    }
  }
}

// Spatial factor of the TRACE problem, Phi(x) = prod_i cos(om_i x_i + be_i)
// with om_i = 1 + i/2, be_i = 0.3 + 0.2 i: its value, gradient and Hessian.
__device__ void trace_phi(int d, const double *x, double *phi, double *dphi, double H[3][3]) {
  double c[3], s[3], om[3];
  for (int i = 0; i < d; ++i) {
    om[i] = 1.0 + 0.5 * i;
    const double a = om[i] * x[i] + 0.3 + 0.2 * i;
    c[i] = cos(a);
    s[i] = sin(a);
  }
  double f = 1.0;
  for (int i = 0; i < d; ++i) f *= c[i];
  *phi = f;
  for (int a = 0; a < d; ++a) {
    double g = -om[a] * s[a];
    for (int i = 0; i < d; ++i)
      if (i != a) g *= c[i];
    dphi[a] = g;
    for (int b = 0; b < d; ++b) {
      double h;
      if (a == b) {
        h = -om[a] * om[a] * f;
      } else {
        h = om[a] * om[b] * s[a] * s[b];
        for (int i = 0; i < d; ++i)
          if (i != a && i != b) h *= c[i];
      }
      H[a][b] = h;
    }
  }
}

// time factor and weights of the TRACE problem's displacement
__device__ inline double trace_T(double t) { return sin(2.0 * t + 0.5); }
__device__ inline double trace_T1(double t) { return 2.0 * cos(2.0 * t + 0.5); }
__device__ inline double trace_T2(double t) { return -4.0 * sin(2.0 * t + 0.5); }
__device__ inline double trace_w(int c) { return c == 0 ? 1.0 : (c == 1 ? -0.7 : 0.4); }

// sum_ab K_ab H_ab over the first d axes (K: 3 x 3 row-major)
__device__ inline double k_contract(int d, const double *K, const double H[3][3]) {
  double v = 0.0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) v += K[a * 3 + b] * H[a][b];
  return v;
}

// Built-in manufactured solutions and their sources
// rho f = rho u_tt - div sigma(u) + alpha grad p,
// g = c0 p_t + alpha div u_t - div(K grad p) (Eq. 1.1), derived by hand, with
// -div(K grad p) = -sum_ab K_ab d_a d_b p for K constant on the cell.  All
// but TRACE vanish on the boundary of the unit box.
__device__ void dev_fields(const ProbDev &P, const double *x, double t, double *u, double *v, double *p) {
  const int d = P.dim;
  for (int i = 0; i < 3; ++i) u[i] = v[i] = 0.0;
  *p = 0.0;
  if (P.id == STFEM_PROBLEM_TRACE) {
    double f, df[3], H[3][3];
    trace_phi(d, x, &f, df, H);
    for (int i = 0; i < d; ++i) {
      u[i] = trace_w(i) * trace_T(t) * f;
      v[i] = trace_w(i) * trace_T1(t) * f;
    }
    *p = cos(t) * f;
  } else if (P.id == STFEM_PROBLEM_SIN) {
    double phi = 1.0;
    for (int i = 0; i < d; ++i) phi *= sin(M_PI * x[i]);
    for (int i = 0; i < d; ++i) {
      u[i] = phi * sin(t);
      v[i] = phi * cos(t);
    }
    *p = phi * cos(t);
  } else if (P.id == STFEM_PROBLEM_PAPER_EOC) {
    const double w1 = M_PI, w2 = M_PI;
    const double T0 = sin(w1 * t * t), T1 = 2.0 * w1 * t * cos(w1 * t * t);
    const double psi = sin(w2 * x[0]) * sin(w2 * x[1]);
    u[0] = u[1] = T0 * psi;
    v[0] = v[1] = T1 * psi;
    *p = T0 * psi;
  } else if (P.id == STFEM_PROBLEM_PAPER_SUPERCONV) {
    const double w1 = 40.0 * M_PI, w2 = 10.0 * M_PI;
    const double X = x[0], Y = x[1];
    const double Ax = X * X * (X - 1) * (X - 1), Ay = Y * Y * (Y - 1) * (Y - 1);
    const double Bx = (X - 1) * X * (2 * X - 1), By = (Y - 1) * Y * (2 * Y - 1);
    u[0] = -2.0 * Ax * By * sin(w1 * t);
    u[1] = 2.0 * Bx * Ay * sin(w1 * t);
    v[0] = -2.0 * Ax * By * w1 * cos(w1 * t);
    v[1] = 2.0 * Bx * Ay * w1 * cos(w1 * t);
    *p = -2.0 * Ax * By * sin(w2 * t);
  }
}

__device__ void dev_source(const ProbDev &P, const double *x, double t, double lam, double mu, const double *K,
                           double *rf, double *g) {
  const int d = P.dim;
  for (int i = 0; i < 3; ++i) rf[i] = 0.0;
  *g = 0.0;
  if (P.id == STFEM_PROBLEM_TRACE) {
    // u_b = w_b T Phi: div sigma(u)_b = mu lap u_b + (mu + lam) d_b div u
    double f, df[3], H[3][3];
    trace_phi(d, x, &f, df, H);
    double lap = 0.0, divw = 0.0;
    for (int a = 0; a < d; ++a) {
      lap += H[a][a];
      divw += trace_w(a) * df[a];
    }
    const double T = trace_T(t), T1 = trace_T1(t), T2 = trace_T2(t);
    for (int b = 0; b < d; ++b) {
      double gd = 0.0; // d_b sum_a w_a d_a Phi
      for (int a = 0; a < d; ++a) gd += trace_w(a) * H[a][b];
      rf[b] = P.rho * trace_w(b) * T2 * f - mu * trace_w(b) * T * lap - (mu + lam) * T * gd +
              P.alpha * cos(t) * df[b];
    }
    *g = -P.c0 * sin(t) * f + P.alpha * T1 * divw - cos(t) * k_contract(d, K, H);
  } else if (P.id == STFEM_PROBLEM_SIN) {
    double s[3], c[3];
    for (int i = 0; i < d; ++i) {
      s[i] = sin(M_PI * x[i]);
      c[i] = cos(M_PI * x[i]);
    }
    double phi = 1.0;
    for (int i = 0; i < d; ++i) phi *= s[i];
    const double pi2 = M_PI * M_PI;
    double dphi[3];
    for (int i = 0; i < d; ++i) {
      double pr = M_PI * c[i];
      for (int k = 0; k < d; ++k)
        if (k != i) pr *= s[k];
      dphi[i] = pr;
    }
    for (int i = 0; i < d; ++i) {
      double hsum = 0.0; // sum_j d_i d_j phi
      for (int j = 0; j < d; ++j) {
        if (j == i) {
          hsum += -pi2 * phi;
        } else {
          double pr = pi2 * c[i] * c[j];
          for (int k = 0; k < d; ++k)
            if (k != i && k != j) pr *= s[k];
          hsum += pr;
        }
      }
      rf[i] = -P.rho * phi * sin(t) + d * pi2 * mu * phi * sin(t) - (mu + lam) * sin(t) * hsum +
              P.alpha * cos(t) * dphi[i];
    }
    double div = 0.0;
    for (int j = 0; j < d; ++j) div += dphi[j];
    double H[3][3]; // Hessian of phi
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        if (i == j) {
          H[i][j] = -pi2 * phi;
        } else {
          double pr = pi2 * c[i] * c[j];
          for (int k = 0; k < d; ++k)
            if (k != i && k != j) pr *= s[k];
          H[i][j] = pr;
        }
      }
    *g = -P.c0 * phi * sin(t) + P.alpha * cos(t) * div - cos(t) * k_contract(d, K, H);
  } else if (P.id == STFEM_PROBLEM_PAPER_EOC) {
    const double w1 = M_PI, w2 = M_PI;
    const double T0 = sin(w1 * t * t), T1 = 2.0 * w1 * t * cos(w1 * t * t),
                 T2 = 2.0 * w1 * cos(w1 * t * t) - 4.0 * w1 * w1 * t * t * sin(w1 * t * t);
    const double sx = sin(w2 * x[0]), sy = sin(w2 * x[1]), cx = cos(w2 * x[0]), cy = cos(w2 * x[1]);
    const double psi = sx * sy, cc = cx * cy, w22 = w2 * w2;
    const double base = P.rho * T2 * psi + 2.0 * mu * w22 * T0 * psi + (mu + lam) * w22 * T0 * (psi - cc);
    rf[0] = base + P.alpha * T0 * w2 * cx * sy;
    rf[1] = base + P.alpha * T0 * w2 * sx * cy;
    const double H[3][3] = {{-w22 * psi, w22 * cc, 0.0}, {w22 * cc, -w22 * psi, 0.0}, {0.0, 0.0, 0.0}};
    *g = P.c0 * T1 * psi + P.alpha * T1 * w2 * (cx * sy + sx * cy) - T0 * k_contract(2, K, H);
  } else if (P.id == STFEM_PROBLEM_PAPER_SUPERCONV) {
    const double w1 = 40.0 * M_PI, w2 = 10.0 * M_PI;
    const double X = x[0], Y = x[1];
    const double Ax = X * X * (X - 1) * (X - 1), Ay = Y * Y * (Y - 1) * (Y - 1);
    const double Bx = (X - 1) * X * (2 * X - 1), By = (Y - 1) * Y * (2 * Y - 1);
    const double A2x = 12 * X * X - 12 * X + 2, A2y = 12 * Y * Y - 12 * Y + 2;
    const double B1y = 6 * Y * Y - 6 * Y + 1, B2x = 12 * X - 6, B2y = 12 * Y - 6;
    const double A1x = 2.0 * Bx; // A' = 2B
    const double s1 = sin(w1 * t), s2 = sin(w2 * t), c2 = cos(w2 * t);
    rf[0] = 2.0 * P.rho * w1 * w1 * Ax * By * s1 + 2.0 * mu * (A2x * By + Ax * B2y) * s1 - 2.0 * P.alpha * A1x * By * s2;
    rf[1] = -2.0 * P.rho * w1 * w1 * Bx * Ay * s1 - 2.0 * mu * (B2x * Ay + Bx * A2y) * s1 - 2.0 * P.alpha * Ax * B1y * s2;
    // p = -2 A(x) B(y) sin(w2 t): Hessian of the spatial factor -2 A B
    const double H[3][3] = {{-2.0 * A2x * By, -2.0 * A1x * B1y, 0.0}, {-2.0 * A1x * B1y, -2.0 * Ax * B2y, 0.0},
                            {0.0, 0.0, 0.0}};
    *g = -2.0 * P.c0 * w2 * Ax * By * c2 - s2 * k_contract(2, K, H);
  }
}

// Gradients of the exact solution (SIN and TRACE): gu[b][a] = d_a u_b,
// gp[a] = d_a p, and p, for the Neumann data of Eq. 3.4.
__device__ void dev_grads(const ProbDev &P, const double *x, double t, double gu[3][3], double *gp, double *p) {
  const int d = P.dim;
  double f = 0.0, df[3] = {0.0, 0.0, 0.0}, tu = 0.0, tp = 0.0, w[3] = {1.0, 1.0, 1.0};
  if (P.id == STFEM_PROBLEM_TRACE) {
    double H[3][3];
    trace_phi(d, x, &f, df, H);
    tu = trace_T(t);
    tp = cos(t);
    for (int c = 0; c < d; ++c) w[c] = trace_w(c);
  } else if (P.id == STFEM_PROBLEM_SIN) {
    double s[3], c[3];
    for (int i = 0; i < d; ++i) {
      s[i] = sin(M_PI * x[i]);
      c[i] = cos(M_PI * x[i]);
    }
    f = 1.0;
    for (int i = 0; i < d; ++i) f *= s[i];
    for (int a = 0; a < d; ++a) {
      double g = M_PI * c[a];
      for (int i = 0; i < d; ++i)
        if (i != a) g *= s[i];
      df[a] = g;
    }
    tu = sin(t);
    tp = cos(t);
  }
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) gu[b][a] = (a < d && b < d) ? w[b] * tu * df[a] : 0.0;
  for (int a = 0; a < 3; ++a) gp[a] = a < d ? tp * df[a] : 0.0;
  *p = tp * f;
}

// z-component of the traction t_N on the top face for the pulse problem
__device__ double dev_top_traction(const ProbDev &P, const double *x, double t) {
  if (P.id != STFEM_PROBLEM_PULSE) return 0.0;
  if (x[0] >= 0.75 && x[0] <= 1.25 && x[1] >= 0.75 && x[1] <= 1.25) return -sin(M_PI * t / 0.05);
  return 0.0;
}

// state = nodal interpolation of (v, u, p) at time t; a broken pressure
// space takes the L2 projection of p on each cell (orthogonal basis: one
// quotient per dof)
__global__ void k_interp(GeomDev g, ProbDev P, LoadTables L, double t, long R, long S, double *__restrict__ state) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * R + S) return;
  double x[3], u[3], v[3], p;
  if (L.pdisc && i >= 2 * R) {
    const long cell = (i - 2 * R) / L.nlp;
    const int s = (int)((i - 2 * R) % L.nlp);
    int cm[3] = {0, 0, 0};
    long t2 = cell;
    for (int k = 0; k < g.dim; ++k) {
      cm[k] = (int)(t2 % g.n[k]);
      t2 /= g.n[k];
    }
    double num = 0.0, den = 0.0;
    for (int qq = 0; qq < L.npq; ++qq) {
      for (int k = 0; k < 3; ++k) x[k] = k < g.dim ? g.lo[k] + g.h[k] * (cm[k] + L.pqx[qq * 3 + k]) : 0.0;
      dev_fields(P, x, t, u, v, &p);
      const double ph = L.phiPP[(long)qq * L.nlp + s];
      num += L.pqw[qq] * p * ph;
      den += L.pqw[qq] * ph * ph;
    }
    state[i] = num / den;
    return;
  }
  if (i < 2 * R) {
    const long rem = i % R;
    node_coord(g, g.r, g.udims, g.refU, rem / g.dim, x);
    dev_fields(P, x, t, u, v, &p);
    state[i] = (i < R) ? v[rem % g.dim] : u[rem % g.dim];
  } else {
    node_coord(g, g.r - 1, g.pdims, g.refP, i - 2 * R, x);
    dev_fields(P, x, t, u, v, &p);
    state[i] = p;
  }
}

// Source values rho f (d components) and g at every (time node b, cell,
// quadrature point) of the finest level: src[((b * ncell + cell) * nq + qp) * 4 + c].
__global__ void k_src_eval(GeomDev g, ProbDev P, LoadTables L, int q, const double *tnode, double t_prev, double tau,
                           long ncell, double *__restrict__ src) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)q * ncell * L.nq) return;
  const int qp = (int)(i % L.nq);
  const long cell = (i / L.nq) % ncell;
  const int b = (int)(i / ((long)L.nq * ncell));
  const double tb = t_prev + 0.5 * tau * (tnode[b] + 1.0);
  long t = cell;
  double x[3];
  for (int k = 0; k < 3; ++k) {
    int c = 0;
    if (k < g.dim) {
      c = (int)(t % g.n[k]);
      t /= g.n[k];
    }
    x[k] = g.lo[k] + g.h[k] * (c + L.qx[qp * 3 + k]);
  }
  double rf[3], gg;
  dev_source(P, x, tb, L.lam[cell], L.mu[cell], L.Kt + cell * 9, rf, &gg);
  double *o = src + i * 4;
  o[0] = rf[0];
  o[1] = rf[1];
  o[2] = rf[2];
  o[3] = gg;
}

// Slab right-hand side (Eq. 3.5 / Eq. 4.5):
// rhs[b, m] = chi_b(-1) (S1 state)[m] + W_b * load_m(t_b), load = 0 on u-rows,
// F = <rho f, psi> - <t_N, psi>_{Gamma_N} on v-rows, G = <g, xi> on p-rows.
// Node-centric gather over the cells holding the node (deterministic), from
// the source values precomputed by k_src_eval.
__global__ void k_rhs(GeomDev g, ProbDev P, LoadTables L, int q, TimeCoef<double> tc, const double *chi,
                      const double *tnode, double t_prev, double tau, long R, long S,
                      const double *__restrict__ src, const double *__restrict__ ys, double *__restrict__ out) {
  const long ns = 2 * R + S;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)q * ns) return;
  const int b = (int)(i / ns);
  const long m = i % ns;
  double val = chi[b] * ys[m];
  if (m >= R && P.id != STFEM_PROBLEM_NONE) {
    const double tb = t_prev + 0.5 * tau * (tnode[b] + 1.0);
    const int d = g.dim;
    const bool urow = m < 2 * R;
    if (!urow && L.pdisc) {
      // broken pressure dof: the load of its own cell alone
      const long ncell = (long)g.n[0] * g.n[1] * g.n[2];
      const long cell = (m - 2 * R) / L.nlp;
      const int li = (int)((m - 2 * R) % L.nlp);
      const double *sv = src + (((long)b * ncell + cell) * L.nq) * 4 + 3;
      double load = 0.0;
      for (int qq = 0; qq < L.nq; ++qq) load += L.qw[qq] * sv[qq * 4] * L.phiP[(long)qq * L.nlp + li];
      out[i] = val + tc.W[b] * load;
      return;
    }
    const int deg = urow ? g.r : g.r - 1;
    const int *dims = urow ? g.udims : g.pdims;
    const long node = urow ? (m - R) / d : m - 2 * R;
    const int comp = urow ? (int)((m - R) % d) : 3;
    int a[3] = {0, 0, 0}, clo[3] = {0, 0, 0}, chi_[3] = {0, 0, 0};
    long t = node;
    for (int k = 0; k < d; ++k) {
      a[k] = (int)(t % dims[k]);
      t /= dims[k];
      if (a[k] % deg == 0) {
        clo[k] = max(a[k] / deg - 1, 0);
        chi_[k] = min(a[k] / deg, g.n[k] - 1);
      } else {
        clo[k] = chi_[k] = a[k] / deg;
      }
    }
    const int nl = urow ? L.nlu : L.nlp;
    const double *phi = urow ? L.phiU : L.phiP;
    const long ncell = (long)g.n[0] * g.n[1] * g.n[2];
    double load = 0.0;
    for (int cz = clo[2]; cz <= chi_[2]; ++cz)
      for (int cy = clo[1]; cy <= chi_[1]; ++cy)
        for (int cx = clo[0]; cx <= chi_[0]; ++cx) {
          const int cc[3] = {cx, cy, cz};
          int li = 0, stride = 1;
          for (int k = 0; k < d; ++k) {
            li += (a[k] - deg * cc[k]) * stride;
            stride *= deg + 1;
          }
          const long cell = cx + (long)g.n[0] * (cy + (long)g.n[1] * cz);
          const double *sv = src + (((long)b * ncell + cell) * L.nq) * 4 + comp;
          for (int qq = 0; qq < L.nq; ++qq) load += L.qw[qq] * sv[qq * 4] * phi[qq * nl + li];
          // Neumann traction on the top face (pulse problem)
          if (urow && L.top_neumann && comp == d - 1 && cc[d - 1] == g.n[d - 1] - 1 &&
              a[d - 1] == deg * g.n[d - 1]) {
            for (int qq = 0; qq < L.nqf; ++qq) {
              double x[3];
              for (int k = 0; k < 3; ++k) x[k] = g.lo[k] + g.h[k] * (cc[k] + L.fx[qq * 3 + k]);
              load += -L.fw[qq] * dev_top_traction(P, x, tb) * L.fphiU[qq * L.nlu + li];
            }
          }
        }
    val += tc.W[b] * load;
  }
  out[i] = val;
}

// Boundary data terms of the loads (Eq. 3.4), added to the slab right-hand
// side at every Radau node t_b (times W_b, as the volume loads):
//   v-rows: -<t_N, psi> on Neumann faces of u; on Dirichlet faces of u the
//           Nitsche terms of a_gamma(u_D, psi): -<u_D, sigma(psi) n>
//           + gamma_a / h_F <u_D, psi>;
//   p-rows: -alpha <v_D . n, xi> on Dirichlet faces of u; -<p_N, xi> on
//           Neumann faces of p; on Dirichlet faces of p the terms of
//           b_gamma(p_D, xi): -<p_D, (K grad xi) . n> + gamma_b / h_F <p_D, xi>;
// and for Problem B.1 the previous-slab data term
// -chi_b(-1) alpha <u_D(t_{n-1}) . n, xi> on Dirichlet faces of u.  One thread
// per (node b, v- or p-row); it visits the cells holding the row's function
// and their faces on the boundary (deterministic).
__global__ void k_rhs_data(GeomDev g, ProbDev P, LoadTables L, int q, TimeCoef<double> tc, const double *chi,
                           const double *tnode, double t_prev, double tau, long R, long S,
                           double *__restrict__ out) {
  const long nrow = R + S, ns = 2 * R + S;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)q * nrow) return;
  const int b = (int)(i / nrow);
  const long m = R + i % nrow;
  const double tb = t_prev + 0.5 * tau * (tnode[b] + 1.0);
  const int d = g.dim;
  const bool vrow = m < 2 * R;
  const bool trace = P.id == STFEM_PROBLEM_TRACE;
  const bool exact_flux = trace || P.id == STFEM_PROBLEM_SIN;
  const int nl = vrow ? L.nlu : L.nlp;
  const int comp = vrow ? (int)((m - R) % d) : 0;
  // the cells holding the row's function: a box of lattice cells, or the
  // dof's own cell for the broken pressure space
  int clo[3] = {0, 0, 0}, chi_[3] = {0, 0, 0}, a[3] = {0, 0, 0};
  int deg = 1;
  long own = -1;
  if (!vrow && L.pdisc) {
    own = (m - 2 * R) / L.nlp;
    long t2 = own;
    for (int k = 0; k < d; ++k) {
      clo[k] = chi_[k] = (int)(t2 % g.n[k]);
      t2 /= g.n[k];
    }
  } else {
    deg = vrow ? g.r : g.r - 1;
    const int *dims = vrow ? g.udims : g.pdims;
    long t2 = vrow ? (m - R) / d : m - 2 * R;
    for (int k = 0; k < d; ++k) {
      a[k] = (int)(t2 % dims[k]);
      t2 /= dims[k];
      if (a[k] % deg == 0) {
        clo[k] = max(a[k] / deg - 1, 0);
        chi_[k] = min(a[k] / deg, g.n[k] - 1);
      } else {
        clo[k] = chi_[k] = a[k] / deg;
      }
    }
  }
  double acc = 0.0, acc0 = 0.0;
  for (int cz = clo[2]; cz <= chi_[2]; ++cz)
    for (int cy = clo[1]; cy <= chi_[1]; ++cy)
      for (int cx = clo[0]; cx <= chi_[0]; ++cx) {
        const int cc[3] = {cx, cy, cz};
        const long cell = cx + (long)g.n[0] * (cy + (long)g.n[1] * cz);
        int li = 0;
        if (own >= 0) {
          li = (int)((m - 2 * R) % L.nlp);
        } else {
          int stride = 1;
          for (int k = 0; k < d; ++k) {
            li += (a[k] - deg * cc[k]) * stride;
            stride *= deg + 1;
          }
        }
        const double lam = L.lam[cell], mu = L.mu[cell];
        for (int f = 0; f < 2 * d; ++f) {
          const int ax = f >> 1, side = f & 1;
          if (cc[ax] != (side ? g.n[ax] - 1 : 0)) continue;
          double n[3] = {0.0, 0.0, 0.0};
          n[ax] = side ? 1.0 : -1.0;
          // (K g) . n = n_ax sum_b K[ax][b] g_b
          const double *Kn = L.Kt + cell * 9 + ax * 3;
          const bool dir_u = P.bc_u[f] == 0, dir_p = P.bc_p[f] == 0;
          if (vrow && (dir_u ? !trace : !exact_flux)) continue;
          if (!vrow && !(dir_u && trace) && (dir_p ? !trace : !exact_flux)) continue;
          for (int qq = 0; qq < L.nqd; ++qq) {
            const long fq = (long)f * L.nqd + qq;
            const double w = L.dfw[fq];
            double x[3];
            for (int k = 0; k < 3; ++k) x[k] = k < d ? g.lo[k] + g.h[k] * (cc[k] + L.dfx[fq * 3 + k]) : 0.0;
            const double *gph = (vrow ? L.dfdU : L.dfdP) + (fq * nl + li) * d;
            const double ph = (vrow ? L.dfU : L.dfP)[fq * nl + li];
            if (vrow) {
              if (!dir_u) {
                double gu[3][3], gp[3], p;
                dev_grads(P, x, tb, gu, gp, &p);
                // t_N[c] = -(sigma(u) n)[c] + alpha p n[c]
                double divu = 0.0, sn = 0.0;
                for (int k = 0; k < d; ++k) divu += gu[k][k];
                for (int k = 0; k < d; ++k) sn += mu * (gu[comp][k] + gu[k][comp]) * n[k];
                sn += lam * divu * n[comp];
                acc += -w * (-sn + P.alpha * p * n[comp]) * ph;
              } else {
                double u[3], v[3], p;
                dev_fields(P, x, tb, u, v, &p);
                // u_D . sigma(psi) n for psi = phi e_comp
                double dn = 0.0, gdu = 0.0, un = 0.0;
                for (int k = 0; k < d; ++k) {
                  dn += gph[k] * n[k];
                  gdu += gph[k] * u[k];
                  un += u[k] * n[k];
                }
                const double usn = mu * (u[comp] * dn + n[comp] * gdu) + lam * gph[comp] * un;
                acc += -w * usn + (P.gam_a / P.hF) * w * u[comp] * ph;
              }
            } else {
              if (dir_u && trace) {
                double u[3], v[3], p;
                dev_fields(P, x, tb, u, v, &p);
                double vn = 0.0;
                for (int k = 0; k < d; ++k) vn += v[k] * n[k];
                acc += -P.alpha * w * vn * ph;
                if (P.b1) {
                  dev_fields(P, x, t_prev, u, v, &p);
                  double un = 0.0;
                  for (int k = 0; k < d; ++k) un += u[k] * n[k];
                  acc0 += -P.alpha * w * un * ph;
                }
              }
              if (!dir_p && exact_flux) {
                double gu[3][3], gp[3], p;
                dev_grads(P, x, tb, gu, gp, &p);
                double pN = 0.0;
                for (int k = 0; k < d; ++k) pN += -n[ax] * Kn[k] * gp[k];
                acc += -w * pN * ph;
              } else if (dir_p && trace) {
                double u[3], v[3], p;
                dev_fields(P, x, tb, u, v, &p);
                double dn = 0.0;
                for (int k = 0; k < d; ++k) dn += n[ax] * Kn[k] * gph[k];
                acc += -w * p * dn + (P.gam_b / P.hF) * w * p * ph;
              }
            }
          }
        }
      }
  out[(long)b * ns + m] += tc.W[b] * acc + chi[b] * acc0;
}
