// Host-side setup of the space-time FE hierarchy (arXiv 2303.06742).
//
// Secs. 2-3: Taylor-Hood Q_r^d / Q_{r-1} spaces on uniform box meshes, the
// forms A_gamma, C, B_gamma with Nitsche terms (Eqs. 3.2-3.3), right
// Gauss-Radau dG(k) in time (Eq. 2.4).  Sec. 4: vertex patches (Eq. 4.9),
// principal-submatrix patch inverses (Def. 4.2, Eq. 4.13), interpolation
// transfers, coarse direct solve.
//
// Readings (the paper is silent or garbled there):
//  * h_F = |K|_d literally (Sec. 3), or |K|_d^{1/d} on request;
//  * gamma_a = 5e4 r (r+1), gamma_b = r (r-1) / 2;
//  * element integrals by Gauss-Legendre with r+2 points per direction;
//  * coarse-level coefficients are the mean of the fine children;
//  * patch dof set: dofs whose basis support lies in the closed patch.
#include "fem.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <atomic>
#include <array>
#include <complex>

namespace stfem {

// ---------------------------------------------------------------- quadrature
static void legendre(int n, double x, double *p, double *dp) {
  // P_n and P_n' by the three-term recurrence and P'_{j+1} = P'_{j-1} + (2j+1) P_j
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  for (int j = 1; j < n; ++j) {
    double p2 = ((2 * j + 1) * x * p1 - j * p0) / (j + 1);
    double d2 = d0 + (2 * j + 1) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *p = p1;
  *dp = d1;
}

Rule gauss01(int n) {
  Rule r;
  r.x.resize(n);
  r.w.resize(n);
  for (int i = 0; i < n; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, x, &p, &dp);
      double dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p, dp;
    legendre(n, x, &p, &dp);
    r.x[n - 1 - i] = 0.5 * (x + 1.0);
    r.w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return r;
}

std::vector<double> lobatto01(int r) {
  std::vector<double> x(r + 1);
  x[0] = -1.0;
  x[r] = 1.0;
  for (int i = 1; i < r; ++i) {
    double z = -std::cos(M_PI * i / r);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(r, z, &p, &dp);
      double d2 = (2.0 * z * dp - r * (r + 1.0) * p) / (1.0 - z * z); // P_r''
      double dz = dp / d2;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (auto &v : x) v = 0.5 * (v + 1.0);
  return x;
}

Rule radau_right(int n) {
  // interior nodes: zeros of P_{n-1} - P_n in (-1, 1) by bracketing and
  // bisection; weights (1 + x) / (n^2 P_{n-1}(x)^2), end weight 2 / n^2.
  Rule r;
  auto f = [n](double x) {
    double a, da, b, db;
    legendre(n - 1, x, &a, &da);
    legendre(n, x, &b, &db);
    return a - b;
  };
  const int M = 20000;
  double xa = -1.0, fa = f(xa);
  for (int i = 1; i <= M && (int)r.x.size() < n - 1; ++i) {
    double xb = -1.0 + 1.999 * i / M, fb = f(xb);
    if (fa == 0.0) {
      r.x.push_back(xa);
    } else if (fa * fb < 0.0) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), fm = f(mid);
        if ((fm < 0) == (flo < 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      r.x.push_back(0.5 * (lo + hi));
    }
    xa = xb;
    fa = fb;
  }
  for (double x : r.x) {
    double a, da;
    legendre(n - 1, x, &a, &da);
    r.w.push_back((1.0 + x) / (double(n) * n * a * a));
  }
  r.x.push_back(1.0);
  r.w.push_back(2.0 / (double(n) * n));
  return r;
}

void lagrange(const std::vector<double> &nodes, double x, double *val, double *der) {
  const int n = (int)nodes.size();
  for (int i = 0; i < n; ++i) {
    double den = 1.0, num = 1.0, d = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      den *= nodes[i] - nodes[j];
      // product rule: d/dx prod_j (x - x_j) = sum_l prod_{j != l} (x - x_j)
      d = d * (x - nodes[j]) + num;
      num *= x - nodes[j];
    }
    val[i] = num / den;
    der[i] = d / den;
  }
}

Temporal make_temporal(int k) {
  Temporal T;
  T.k = k;
  T.q = k + 1;
  Rule r = radau_right(T.q);
  T.t = r.x;
  T.w = r.w;
  T.chi_m1.resize(T.q);
  std::vector<double> v(T.q), d(T.q);
  lagrange(T.t, -1.0, T.chi_m1.data(), d.data());
  T.Dt.assign(T.q * T.q, 0.0);
  for (int b = 0; b < T.q; ++b) {
    lagrange(T.t, T.t[b], v.data(), d.data());
    for (int a = 0; a < T.q; ++a)
      T.Dt[b * T.q + a] = T.w[b] * d[a] + T.chi_m1[a] * T.chi_m1[b];
  }
  return T;
}

// ---------------------------------------------------------------- mesh
Box make_box(int dim, const double *lo, const double *hi, const int *n, int hf_mode) {
  Box b;
  b.dim = dim;
  b.vol = 1.0;
  b.ncell = 1;
  for (int i = 0; i < 3; ++i) {
    b.lo[i] = i < dim ? lo[i] : 0.0;
    b.hi[i] = i < dim ? hi[i] : 1.0;
    b.n[i] = i < dim ? n[i] : 1;
    b.h[i] = (b.hi[i] - b.lo[i]) / b.n[i];
    if (i < dim) {
      b.vol *= b.h[i];
      b.ncell *= b.n[i];
    }
  }
  b.hF = hf_mode == 1 ? std::pow(b.vol, 1.0 / dim) : b.vol;
  return b;
}

Coef coarsen(const Coef &f, const Box &fb) {
  Coef c;
  c.rho = f.rho;
  c.alpha = f.alpha;
  c.c0 = f.c0;
  int nc[3] = {1, 1, 1};
  for (int i = 0; i < fb.dim; ++i) nc[i] = fb.n[i] / 2;
  long ncc = (long)nc[0] * nc[1] * nc[2];
  c.lam.assign(ncc, 0.0);
  c.mu.assign(ncc, 0.0);
  c.kap.assign(ncc, 0.0);
  const int dd = fb.dim * fb.dim;
  if (!f.K.empty()) c.K.assign((size_t)ncc * dd, 0.0);
  const int nchild = 1 << fb.dim;
  for (int z = 0; z < nc[2]; ++z)
    for (int y = 0; y < nc[1]; ++y)
      for (int x = 0; x < nc[0]; ++x) {
        long ci = x + (long)nc[0] * (y + (long)nc[1] * z);
        for (int ch = 0; ch < nchild; ++ch) {
          int fx = 2 * x + (ch & 1), fy = fb.dim > 1 ? 2 * y + ((ch >> 1) & 1) : 0,
              fz = fb.dim > 2 ? 2 * z + ((ch >> 2) & 1) : 0;
          long fi = fx + (long)fb.n[0] * (fy + (long)fb.n[1] * fz);
          c.lam[ci] += f.lam[fi] / nchild;
          c.mu[ci] += f.mu[fi] / nchild;
          c.kap[ci] += f.kap[fi] / nchild;
          if (!f.K.empty())
            for (int e = 0; e < dd; ++e) c.K[(size_t)ci * dd + e] += f.K[(size_t)fi * dd + e] / nchild;
        }
      }
  return c;
}

Lattice make_lattice(const Box &b, int m) {
  Lattice L;
  L.dim = b.dim;
  L.m = m;
  L.nnodes = 1;
  for (int i = 0; i < 3; ++i) {
    L.dims[i] = i < b.dim ? m * b.n[i] + 1 : 1;
    L.nnodes *= L.dims[i];
  }
  L.ref = lobatto01(m);
  return L;
}

void cells_of(int a, int m, int ncell, int *c_lo, int *c_hi) {
  if (a % m == 0) {
    *c_lo = std::max(a / m - 1, 0);
    *c_hi = std::min(a / m, ncell - 1);
  } else {
    *c_lo = *c_hi = a / m;
  }
}

// ---------------------------------------------------------------- assembly
namespace {

inline void unflatten(long idx, const int *dims, int dim, int *a) {
  for (int i = 0; i < 3; ++i) {
    if (i < dim) {
      a[i] = (int)(idx % dims[i]);
      idx /= dims[i];
    } else {
      a[i] = 0;
    }
  }
}

inline long flatten(const int *a, const int *dims) {
  return a[0] + (long)dims[0] * (a[1] + (long)dims[1] * a[2]);
}

// Neighbour box of a node (lattice coordinate a with degree m_row) inside the
// lattice of degree m_col: the nodes of all cells holding the node.
struct NbrBox {
  int lo[3], ext[3];
  long size;
};

inline NbrBox nbr_box(const int *a, int m_row, int m_col, const Box &b) {
  NbrBox nb;
  nb.size = 1;
  for (int i = 0; i < 3; ++i) {
    if (i < b.dim) {
      int clo, chi;
      cells_of(a[i], m_row, b.n[i], &clo, &chi);
      nb.lo[i] = m_col * clo;
      nb.ext[i] = m_col * (chi + 1) - nb.lo[i] + 1;
    } else {
      nb.lo[i] = 0;
      nb.ext[i] = 1;
    }
    nb.size *= nb.ext[i];
  }
  return nb;
}

inline long nbr_pos(const NbrBox &nb, const int *a) {
  return (a[0] - nb.lo[0]) + (long)nb.ext[0] * ((a[1] - nb.lo[1]) + (long)nb.ext[1] * (a[2] - nb.lo[2]));
}

// Node-level matrix with a fixed number of values per entry.
struct NodeMat {
  std::vector<long> rowptr;
  hvec<double> val; // nvals per entry
  int nvals = 1;
};

NodeMat make_nodemat(const Lattice &row, const Lattice &colL, const Box &b, int nvals) {
  NodeMat M;
  M.nvals = nvals;
  M.rowptr.resize(row.nnodes + 1);
  M.rowptr[0] = 0;
  int a[3];
  for (long i = 0; i < row.nnodes; ++i) {
    unflatten(i, row.dims, b.dim, a);
    M.rowptr[i + 1] = M.rowptr[i] + nbr_box(a, row.m, colL.m, b).size;
  }
  const long nv = M.rowptr[row.nnodes] * nvals;
  M.val.resize(nv);
  double *v = M.val.data();
#pragma omp parallel for schedule(static)
  for (long i = 0; i < nv; ++i) v[i] = 0.0;
  return M;
}

// Tensor-product reference data of one scalar space at a set of points.
struct RefData {
  int nloc = 0, npts = 0, dim = 2;
  std::vector<double> phi;  // [pt][loc]
  std::vector<double> dphi; // [pt][loc][dim], physical derivatives
  std::vector<int> loc;     // [loc][3] local lattice offsets
};

RefData ref_data(const Lattice &L, const Box &b, const std::vector<std::array<double, 3>> &pts) {
  RefData R;
  R.dim = b.dim;
  const int m1 = L.m + 1;
  R.nloc = 1;
  for (int i = 0; i < b.dim; ++i) R.nloc *= m1;
  R.npts = (int)pts.size();
  R.loc.resize(R.nloc * 3);
  for (int l = 0; l < R.nloc; ++l) {
    int t = l;
    for (int i = 0; i < 3; ++i) {
      if (i < b.dim) {
        R.loc[l * 3 + i] = t % m1;
        t /= m1;
      } else {
        R.loc[l * 3 + i] = 0;
      }
    }
  }
  R.phi.assign((size_t)R.npts * R.nloc, 0.0);
  R.dphi.assign((size_t)R.npts * R.nloc * b.dim, 0.0);
  std::vector<double> v(m1), d(m1);
  for (int q = 0; q < R.npts; ++q) {
    double vals[3][16] = {}, ders[3][16] = {};
    for (int i = 0; i < b.dim; ++i) {
      lagrange(L.ref, pts[q][i], v.data(), d.data());
      for (int j = 0; j < m1; ++j) {
        vals[i][j] = v[j];
        ders[i][j] = d[j] / b.h[i];
      }
    }
    for (int l = 0; l < R.nloc; ++l) {
      double p = 1.0;
      for (int i = 0; i < b.dim; ++i) p *= vals[i][R.loc[l * 3 + i]];
      R.phi[(size_t)q * R.nloc + l] = p;
      for (int j = 0; j < b.dim; ++j) {
        double g = 1.0;
        for (int i = 0; i < b.dim; ++i) g *= (i == j) ? ders[i][R.loc[l * 3 + i]] : vals[i][R.loc[l * 3 + i]];
        R.dphi[((size_t)q * R.nloc + l) * b.dim + j] = g;
      }
    }
  }
  return R;
}

// Exponents of the broken P_m basis: total degree <= m, x exponent fastest.
std::vector<std::array<int, 3>> disc_exponents(int m, int dim) {
  std::vector<std::array<int, 3>> e;
  const int ez = dim > 2 ? m : 0, ey = dim > 1 ? m : 0;
  for (int z = 0; z <= ez; ++z)
    for (int y = 0; y <= ey; ++y)
      for (int x = 0; x <= m; ++x)
        if (x + y + z <= m) e.push_back({x, y, z});
  return e;
}

// Reference data of the broken P_m space: products of Legendre polynomials
// L_a(2 xi - 1) of the reference coordinates.
RefData ref_data_disc(int m, const Box &b, const std::vector<std::array<double, 3>> &pts) {
  RefData R;
  R.dim = b.dim;
  const auto ex = disc_exponents(m, b.dim);
  R.nloc = (int)ex.size();
  R.npts = (int)pts.size();
  R.loc.assign(R.nloc * 3, 0);
  R.phi.assign((size_t)R.npts * R.nloc, 0.0);
  R.dphi.assign((size_t)R.npts * R.nloc * b.dim, 0.0);
  for (int q = 0; q < R.npts; ++q) {
    double vals[3][16] = {}, ders[3][16] = {};
    for (int i = 0; i < b.dim; ++i)
      for (int a = 0; a <= m; ++a) {
        double p, dp;
        legendre(a, 2.0 * pts[q][i] - 1.0, &p, &dp);
        vals[i][a] = p;
        ders[i][a] = 2.0 * dp / b.h[i];
      }
    for (int l = 0; l < R.nloc; ++l) {
      double v = 1.0;
      for (int i = 0; i < b.dim; ++i) v *= vals[i][ex[l][i]];
      R.phi[(size_t)q * R.nloc + l] = v;
      for (int j = 0; j < b.dim; ++j) {
        double g = 1.0;
        for (int i = 0; i < b.dim; ++i) g *= (i == j) ? ders[i][ex[l][i]] : vals[i][ex[l][i]];
        R.dphi[((size_t)q * R.nloc + l) * b.dim + j] = g;
      }
    }
  }
  return R;
}

std::vector<std::array<double, 3>> cell_points(const Box &b, int nq, std::vector<double> *w) {
  Rule g = gauss01(nq);
  std::vector<std::array<double, 3>> pts;
  w->clear();
  int nz = b.dim > 2 ? nq : 1, ny = b.dim > 1 ? nq : 1;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nq; ++x) {
        pts.push_back({g.x[x], b.dim > 1 ? g.x[y] : 0.0, b.dim > 2 ? g.x[z] : 0.0});
        double ww = g.w[x] * (b.dim > 1 ? g.w[y] : 1.0) * (b.dim > 2 ? g.w[z] : 1.0);
        w->push_back(ww * b.vol);
      }
  return pts;
}

std::vector<std::array<double, 3>> face_points(const Box &b, int nq, int ax, int side,
                                               std::vector<double> *w) {
  Rule g = gauss01(nq);
  std::vector<std::array<double, 3>> pts;
  w->clear();
  int other[2], no = 0;
  for (int i = 0; i < b.dim; ++i)
    if (i != ax) other[no++] = i;
  double area = b.vol / b.h[ax];
  int n1 = no > 1 ? nq : 1;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < nq; ++i) {
      std::array<double, 3> p = {0, 0, 0};
      p[ax] = side;
      p[other[0]] = g.x[i];
      if (no > 1) p[other[1]] = g.x[j];
      pts.push_back(p);
      w->push_back(g.w[i] * (no > 1 ? g.w[j] : 1.0) * area);
    }
  return pts;
}

struct Entry {
  int col;
  double v1, v2;
};

// Spatial system CSR of a level with the broken pressure space.  u- and
// v-rows take the node-level UU values; the pressure couplings come from the
// cell-private blocks (C per cell: np x du; (Mp, B) per cell: np x np pairs)
// and the interior penalty faces between neighbouring cells.
void expand_disc(Level &L, const NodeMat &UU, const std::vector<double> &cellC, const std::vector<double> &cellMB,
                 const RefData &RU, double gam, bool b1) {
  const Box &b = L.box;
  const int d = b.dim, r = L.r, np = L.pnloc, nu = RU.nloc, du = nu * d;
  const double rho = L.coef.rho, c0 = L.coef.c0;
  const long R = L.R, ns = L.ns;
  std::vector<std::vector<Entry>> rows(ns);
  // reference data of the broken basis on both sides of a face, per axis
  struct FaceRef {
    RefData a, b;
    std::vector<double> w;
  };
  std::vector<FaceRef> fr(d);
  for (int ax = 0; ax < d; ++ax) {
    std::vector<double> wa, wb;
    auto pa = face_points(b, r + 2, ax, 1, &wa); // on K+ (the lower cell's upper face)
    auto pb = face_points(b, r + 2, ax, 0, &wb); // on K- (the upper cell's lower face)
    fr[ax].a = ref_data_disc(r - 1, b, pa);
    fr[ax].b = ref_data_disc(r - 1, b, pb);
    fr[ax].w = wa;
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (long row = 0; row < ns; ++row) {
    std::vector<Entry> &E = rows[row];
    int a[3];
    if (row < 2 * R) {
      const bool vrow = row >= R;
      const long I = (row % R) / d;
      const int c = (int)((row % R) % d);
      unflatten(I, L.U.dims, d, a);
      NbrBox nbu = nbr_box(a, r, r, b);
      const double *uu = &UU.val[UU.rowptr[I] * UU.nvals];
      long t = 0;
      for (int z = 0; z < nbu.ext[2]; ++z)
        for (int y = 0; y < nbu.ext[1]; ++y)
          for (int x = 0; x < nbu.ext[0]; ++x, ++t) {
            int aj[3] = {nbu.lo[0] + x, nbu.lo[1] + y, nbu.lo[2] + z};
            const long J = flatten(aj, L.U.dims);
            const double m = uu[t * UU.nvals];
            if (!vrow) {
              E.push_back({(int)(J * d + c), 0.0, -rho * m});
              E.push_back({(int)(R + J * d + c), rho * m, 0.0});
            } else {
              E.push_back({(int)(J * d + c), rho * m, 0.0});
              for (int cp = 0; cp < d; ++cp) E.push_back({(int)(R + J * d + cp), 0.0, uu[t * UU.nvals + 1 + c * d + cp]});
            }
          }
      if (vrow) {
        // C^T from every cell holding node I
        int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i) cells_of(a[i], r, b.n[i], &clo[i], &chi[i]);
        for (int cz = clo[2]; cz <= chi[2]; ++cz)
          for (int cy = clo[1]; cy <= chi[1]; ++cy)
            for (int cx = clo[0]; cx <= chi[0]; ++cx) {
              const int cc[3] = {cx, cy, cz};
              int l = 0, stride = 1;
              for (int i = 0; i < d; ++i) {
                l += (a[i] - r * cc[i]) * stride;
                stride *= r + 1;
              }
              const long cell = flatten(cc, b.n);
              const double *Cc = cellC.data() + (size_t)cell * np * du;
              for (int s2 = 0; s2 < np; ++s2) E.push_back({(int)(2 * R + cell * np + s2), 0.0, Cc[s2 * du + l * d + c]});
            }
      }
    } else {
      const long sI = row - 2 * R, cell = sI / np;
      const int s2 = (int)(sI % np);
      int cm[3];
      unflatten(cell, b.n, d, cm);
      const double *Cc = cellC.data() + (size_t)cell * np * du;
      for (int j = 0; j < nu; ++j) {
        int aj[3];
        for (int i = 0; i < 3; ++i) aj[i] = i < d ? r * cm[i] + RU.loc[j * 3 + i] : 0;
        const long J = flatten(aj, L.U.dims);
        for (int cp = 0; cp < d; ++cp) {
          const double v = -Cc[s2 * du + j * d + cp];
          if (b1)
            E.push_back({(int)(R + J * d + cp), v, 0.0});
          else
            E.push_back({(int)(J * d + cp), 0.0, v});
        }
      }
      const double *mb = cellMB.data() + (size_t)cell * np * np * 2;
      for (int t2 = 0; t2 < np; ++t2)
        E.push_back({(int)(2 * R + cell * np + t2), c0 * mb[2 * (s2 * np + t2)], mb[2 * (s2 * np + t2) + 1]});
      // interior faces of this cell: as K+ (neighbour above) and as K- (below)
      for (int ax = 0; ax < d; ++ax)
        for (int side = 0; side < 2; ++side) {
          int cn[3] = {cm[0], cm[1], cm[2]};
          cn[ax] += side ? 1 : -1;
          if (cn[ax] < 0 || cn[ax] >= b.n[ax]) continue;
          const long nb_cell = flatten(cn, b.n);
          const long lower = side ? cell : nb_cell, upper = side ? nb_cell : cell;
          // (K grad psi) . e_ax = sum_b K[ax][b] d_b psi on either side
          const double ka = L.coef.kap[lower], kb = L.coef.kap[upper];
          const double *Ka = L.coef.K.empty() ? nullptr : &L.coef.K[(size_t)lower * d * d + ax * d];
          const double *Kb = L.coef.K.empty() ? nullptr : &L.coef.K[(size_t)upper * d * d + ax * d];
          auto kflux = [&](const double *g, const double *Krow, double kap) {
            if (!Krow) return kap * g[ax];
            double v = 0.0;
            for (int bb = 0; bb < d; ++bb) v += Krow[bb] * g[bb];
            return v;
          };
          const FaceRef &F = fr[ax];
          const int nq = F.a.npts;
          // this row's test function is in the lower (side 1) or upper cell
          for (int q = 0; q < nq; ++q) {
            const double W = F.w[q];
            const double *pa = &F.a.phi[(size_t)q * np], *pb = &F.b.phi[(size_t)q * np];
            const double *ga = &F.a.dphi[(size_t)q * np * d], *gb = &F.b.dphi[(size_t)q * np * d];
            // test values: jump and flux average of psi_row
            const double jr = side ? pa[s2] : -pb[s2];
            const double fr_ = side ? 0.5 * kflux(&ga[s2 * d], Ka, ka) : 0.5 * kflux(&gb[s2 * d], Kb, kb);
            for (int t2 = 0; t2 < np; ++t2) {
              // trial functions of the lower cell, then of the upper cell
              const double js[2] = {pa[t2], -pb[t2]};
              const double fs[2] = {0.5 * kflux(&ga[t2 * d], Ka, ka), 0.5 * kflux(&gb[t2 * d], Kb, kb)};
              const long cl[2] = {lower, upper};
              for (int k = 0; k < 2; ++k) {
                const double v = W * (-fs[k] * jr - js[k] * fr_ + (gam / b.hF) * js[k] * jr);
                E.push_back({(int)(2 * R + cl[k] * np + t2), 0.0, v});
              }
            }
          }
        }
    }
    // merge duplicate columns (the own-cell block meets the face blocks)
    std::sort(E.begin(), E.end(), [](const Entry &x, const Entry &y) { return x.col < y.col; });
    size_t o = 0;
    for (size_t i = 0; i < E.size(); ++i) {
      if (o > 0 && E[o - 1].col == E[i].col) {
        E[o - 1].v1 += E[i].v1;
        E[o - 1].v2 += E[i].v2;
      } else {
        E[o++] = E[i];
      }
    }
    E.resize(o);
  }
  L.rowptr.assign(ns + 1, 0);
  for (long i = 0; i < ns; ++i) L.rowptr[i + 1] = L.rowptr[i] + (int)rows[i].size();
  const long nnz = L.rowptr[ns];
  L.col.resize(nnz);
  L.v1.resize(nnz);
  L.v2.resize(nnz);
#pragma omp parallel for schedule(dynamic, 256)
  for (long i = 0; i < ns; ++i) {
    long e = L.rowptr[i];
    for (const Entry &x : rows[i]) {
      L.col[e] = x.col;
      L.v1[e] = x.v1;
      L.v2[e] = x.v2;
      ++e;
    }
  }
}

} // namespace

void face_tables(const Level &L, FaceTables *out) {
  const Box &b = L.box;
  const int d = b.dim, r = L.r;
  FaceTables &T = *out;
  T = FaceTables();
  for (int f = 0; f < 2 * d; ++f) {
    std::vector<double> w;
    auto pts = face_points(b, r + 2, f / 2, f % 2, &w);
    RefData FU = ref_data(L.U, b, pts), FP = L.pdisc ? ref_data_disc(r - 1, b, pts) : ref_data(L.P, b, pts);
    T.npts = (int)pts.size();
    T.nu = FU.nloc;
    T.np = FP.nloc;
    for (const auto &x : pts) T.x.insert(T.x.end(), x.begin(), x.end());
    T.w.insert(T.w.end(), w.begin(), w.end());
    T.U.insert(T.U.end(), FU.phi.begin(), FU.phi.end());
    T.dU.insert(T.dU.end(), FU.dphi.begin(), FU.dphi.end());
    T.P.insert(T.P.end(), FP.phi.begin(), FP.phi.end());
    T.dP.insert(T.dP.end(), FP.dphi.begin(), FP.dphi.end());
  }
}

Level assemble_level(const Box &b, int r, const Coef &coef, const BCs &bc, int form, int pressure) {
  Level L;
  L.form = form;
  L.box = b;
  L.r = r;
  L.coef = coef;
  L.U = make_lattice(b, r);
  const int d = b.dim;
  const bool disc = pressure == STFEM_PRESSURE_BROKEN;
  L.pdisc = disc;
  if (disc) {
    L.pnloc = (int)disc_exponents(r - 1, d).size();
    L.P = Lattice();
    L.P.dim = d;
    L.P.m = r - 1;
    L.P.nnodes = b.ncell * L.pnloc;
  } else {
    L.P = make_lattice(b, r - 1);
  }
  L.R = (long)d * L.U.nnodes;
  L.S = L.P.nnodes;
  L.ns = 2 * L.R + L.S;
  const double gam_a = 5.0e4 * r * (r + 1), gam_b = 0.5 * r * (r - 1);
  const double alpha = coef.alpha;

  // reference element data
  std::vector<double> wq;
  auto pts = cell_points(b, r + 2, &wq);
  RefData RU = ref_data(L.U, b, pts), RP = disc ? ref_data_disc(r - 1, b, pts) : ref_data(L.P, b, pts);
  const int nu = RU.nloc, np = RP.nloc, nq = RU.npts, du = nu * d;
  // unit-coefficient element matrices
  std::vector<double> Mu(nu * nu, 0), Kmu(du * du, 0), Klam(du * du, 0), Cv(np * du, 0), Bv(np * np, 0),
      Mp(np * np, 0);
  for (int q = 0; q < nq; ++q) {
    const double W = wq[q];
    const double *pu = &RU.phi[(size_t)q * nu], *gu = &RU.dphi[(size_t)q * nu * d];
    const double *pp = &RP.phi[(size_t)q * np], *gp = &RP.dphi[(size_t)q * np * d];
    for (int i = 0; i < nu; ++i)
      for (int j = 0; j < nu; ++j) {
        Mu[i * nu + j] += W * pu[i] * pu[j];
        double gg = 0;
        for (int a = 0; a < d; ++a) gg += gu[i * d + a] * gu[j * d + a];
        for (int c = 0; c < d; ++c)
          for (int cp = 0; cp < d; ++cp) {
            int I = i * d + c, J = j * d + cp;
            Kmu[I * du + J] += W * ((c == cp ? gg : 0.0) + gu[j * d + c] * gu[i * d + cp]);
            Klam[I * du + J] += W * gu[i * d + c] * gu[j * d + cp];
          }
      }
    for (int s = 0; s < np; ++s)
      for (int j = 0; j < nu; ++j)
        for (int cp = 0; cp < d; ++cp) Cv[s * du + j * d + cp] += -alpha * W * gu[j * d + cp] * pp[s];
    for (int rr = 0; rr < np; ++rr)
      for (int s = 0; s < np; ++s) {
        double gg = 0;
        for (int a = 0; a < d; ++a) gg += gp[s * d + a] * gp[rr * d + a];
        Bv[rr * np + s] += W * gg;
        Mp[rr * np + s] += W * pp[rr] * pp[s];
      }
  }
  // a permeability tensor per cell: (K grad psi_s, grad psi_r) =
  // sum_ab K_ab BvK[a d + b], BvK[a d + b][r][s] = (d_b psi_s, d_a psi_r)
  const bool ktensor = !coef.K.empty();
  std::vector<double> BvK;
  if (ktensor) {
    BvK.assign((size_t)d * d * np * np, 0.0);
    for (int q = 0; q < nq; ++q) {
      const double W = wq[q];
      const double *gp = &RP.dphi[(size_t)q * np * d];
      for (int a = 0; a < d; ++a)
        for (int bb = 0; bb < d; ++bb)
          for (int rr = 0; rr < np; ++rr)
            for (int s = 0; s < np; ++s)
              BvK[((size_t)(a * d + bb) * np + rr) * np + s] += W * gp[s * d + bb] * gp[rr * d + a];
    }
  }
  // face matrices, per face id
  // BK[b] (tensor K only): the face consistency terms of B_gamma split by
  // the derivative direction b: with n = +-e_ax, (K grad psi) . n =
  // n_ax sum_b K[ax][b] d_b psi, so the terms are sum_b K[ax][b] BK[b]
  struct FaceMats {
    std::vector<double> Kmu, Klam, Kpen, C, B, Bpen;
    std::vector<double> BK[3];
  };
  std::vector<FaceMats> F(2 * d);
  for (int ax = 0; ax < d; ++ax)
    for (int side = 0; side < 2; ++side) {
      FaceMats &fm = F[2 * ax + side];
      fm.Kmu.assign(du * du, 0);
      fm.Klam.assign(du * du, 0);
      fm.Kpen.assign(du * du, 0);
      fm.C.assign(np * du, 0);
      fm.B.assign(np * np, 0);
      fm.Bpen.assign(np * np, 0);
      std::vector<double> wf;
      auto fp = face_points(b, r + 2, ax, side, &wf);
      RefData FU = ref_data(L.U, b, fp), FP = disc ? ref_data_disc(r - 1, b, fp) : ref_data(L.P, b, fp);
      double n[3] = {0, 0, 0};
      n[ax] = side ? 1.0 : -1.0;
      for (int q = 0; q < (int)fp.size(); ++q) {
        const double W = wf[q];
        const double *pu = &FU.phi[(size_t)q * nu], *gu = &FU.dphi[(size_t)q * nu * d];
        const double *pp = &FP.phi[(size_t)q * np], *gp = &FP.dphi[(size_t)q * np * d];
        for (int i = 0; i < nu; ++i) {
          double dni = 0;
          for (int a = 0; a < d; ++a) dni += gu[i * d + a] * n[a];
          for (int j = 0; j < nu; ++j) {
            double dnj = 0;
            for (int a = 0; a < d; ++a) dnj += gu[j * d + a] * n[a];
            for (int c = 0; c < d; ++c)
              for (int cp = 0; cp < d; ++cp) {
                int I = i * d + c, J = j * d + cp;
                double delta = (c == cp) ? 1.0 : 0.0;
                // -<sigma(psi_J) n, psi_I> - <psi_J, sigma(psi_I) n>
                fm.Kmu[I * du + J] += -W * pu[i] * (delta * dnj + gu[j * d + c] * n[cp]) -
                                      W * pu[j] * (delta * dni + gu[i * d + cp] * n[c]);
                fm.Klam[I * du + J] += -W * pu[i] * gu[j * d + cp] * n[c] - W * pu[j] * gu[i * d + c] * n[cp];
                fm.Kpen[I * du + J] += delta * (gam_a / b.hF) * W * pu[i] * pu[j];
              }
          }
        }
        for (int s = 0; s < np; ++s)
          for (int j = 0; j < nu; ++j)
            for (int cp = 0; cp < d; ++cp) fm.C[s * du + j * d + cp] += alpha * W * pu[j] * n[cp] * pp[s];
        for (int rr = 0; rr < np; ++rr) {
          double dnr = 0;
          for (int a = 0; a < d; ++a) dnr += gp[rr * d + a] * n[a];
          for (int s = 0; s < np; ++s) {
            double dns = 0;
            for (int a = 0; a < d; ++a) dns += gp[s * d + a] * n[a];
            fm.B[rr * np + s] += -W * (dns * pp[rr] + pp[s] * dnr);
            fm.Bpen[rr * np + s] += (gam_b / b.hF) * W * pp[s] * pp[rr];
            if (ktensor)
              for (int bb = 0; bb < d; ++bb) {
                if (fm.BK[bb].empty()) fm.BK[bb].assign((size_t)np * np, 0.0);
                fm.BK[bb][rr * np + s] += -W * n[ax] * (gp[s * d + bb] * pp[rr] + pp[s] * gp[rr * d + bb]);
              }
          }
        }
      }
    }

  L.bc = bc;
  if (!disc) {
    Level::Elem &E = L.elem;
    E.nu = nu;
    E.np = np;
    E.locu = RU.loc;
    E.locp = RP.loc;
    E.Mu = Mu;
    E.Kmu = Kmu;
    E.Klam = Klam;
    E.Cv = Cv;
    E.Bv = Bv;
    E.Mp = Mp;
    for (int f = 0; f < 2 * d; ++f) {
      E.fKmu[f] = F[f].Kmu;
      E.fKlam[f] = F[f].Klam;
      E.fKpen[f] = F[f].Kpen;
      E.fC[f] = F[f].C;
      E.fB[f] = F[f].B;
      E.fBpen[f] = F[f].Bpen;
    }
  }

  // node-level matrices
  NodeMat UU = make_nodemat(L.U, L.U, b, 1 + d * d); // M, K[c][c']
  NodeMat UP, PU, PP;                               // C^T: C[s][(I,c)]; C[s][(J,c')]; Mp, B
  const bool b1 = form == STFEM_FORM_PROBLEM_B_1;
  NodeMat PUv; // volume part of C (Problem B.1 only)
  // broken pressure space: the cell-local blocks C (np x du) and (Mp, B)
  std::vector<double> cellC, cellMB;
  if (disc) {
    cellC.assign((size_t)b.ncell * np * du, 0.0);
    cellMB.assign((size_t)b.ncell * np * np * 2, 0.0);
  } else {
    UP = make_nodemat(L.U, L.P, b, d);
    PU = make_nodemat(L.P, L.U, b, d);
    PP = make_nodemat(L.P, L.P, b, 2);
    if (b1) PUv = make_nodemat(L.P, L.U, b, d);
  }
  // cells in 2^d colour classes by the parity of their coordinates: cells of
  // one class share no node, so a class is scattered in parallel
  std::vector<std::vector<long>> colour(1 << d);
  {
    int cc[3];
    for (long c = 0; c < b.ncell; ++c) {
      unflatten(c, b.n, d, cc);
      int k = 0;
      for (int i = 0; i < d; ++i) k |= (cc[i] & 1) << i;
      colour[k].push_back(c);
    }
  }
  for (const std::vector<long> &cells : colour) {
#pragma omp parallel
  {
  std::vector<double> Ke(du * du), Ce(np * du), Be(np * np);
  int cm[3];
#pragma omp for schedule(dynamic, 16)
  for (long ci = 0; ci < (long)cells.size(); ++ci) {
    const long c = cells[ci];
    unflatten(c, b.n, d, cm);
    const double lam = coef.lam[c], mu = coef.mu[c], kap = coef.kap[c];
    const double *Kc = ktensor ? &coef.K[(size_t)c * d * d] : nullptr;
    for (int i = 0; i < du * du; ++i) Ke[i] = lam * Klam[i] + mu * Kmu[i];
    for (int i = 0; i < np * du; ++i) Ce[i] = Cv[i];
    if (Kc) {
      for (int i = 0; i < np * np; ++i) {
        double v = 0.0;
        for (int e = 0; e < d * d; ++e) v += Kc[e] * BvK[(size_t)e * np * np + i];
        Be[i] = v;
      }
    } else {
      for (int i = 0; i < np * np; ++i) Be[i] = kap * Bv[i];
    }
    for (int ax = 0; ax < d; ++ax)
      for (int side = 0; side < 2; ++side) {
        bool on = side ? (cm[ax] == b.n[ax] - 1) : (cm[ax] == 0);
        if (!on) continue;
        int f = 2 * ax + side;
        if (bc.bc_u[f] == 0) {
          for (int i = 0; i < du * du; ++i) Ke[i] += lam * F[f].Klam[i] + mu * F[f].Kmu[i] + F[f].Kpen[i];
          for (int i = 0; i < np * du; ++i) Ce[i] += F[f].C[i];
        }
        if (bc.bc_p[f] == 0) {
          if (Kc) {
            for (int i = 0; i < np * np; ++i) {
              double v = F[f].Bpen[i];
              for (int bb = 0; bb < d; ++bb) v += Kc[ax * d + bb] * F[f].BK[bb][i];
              Be[i] += v;
            }
          } else {
            for (int i = 0; i < np * np; ++i) Be[i] += kap * F[f].B[i] + F[f].Bpen[i];
          }
        }
      }
    // global lattice coordinates of local nodes
    int gu_[216][3], gp_[216][3];
    long giu[216], gip[216];
    for (int l = 0; l < nu; ++l) {
      for (int i = 0; i < 3; ++i) gu_[l][i] = (i < d) ? r * cm[i] + RU.loc[l * 3 + i] : 0;
      giu[l] = flatten(gu_[l], L.U.dims);
    }
    if (!disc)
      for (int l = 0; l < np; ++l) {
        for (int i = 0; i < 3; ++i) gp_[l][i] = (i < d) ? (r - 1) * cm[i] + RP.loc[l * 3 + i] : 0;
        gip[l] = flatten(gp_[l], L.P.dims);
      }
    for (int i = 0; i < nu; ++i) {
      NbrBox nbu = nbr_box(gu_[i], r, r, b);
      for (int j = 0; j < nu; ++j) {
        long e = UU.rowptr[giu[i]] + nbr_pos(nbu, gu_[j]);
        double *v = &UU.val[e * UU.nvals];
        v[0] += Mu[i * nu + j];
        for (int c = 0; c < d; ++c)
          for (int cp = 0; cp < d; ++cp) v[1 + c * d + cp] += Ke[(i * d + c) * du + j * d + cp];
      }
      if (disc) continue;
      NbrBox nbp = nbr_box(gu_[i], r, r - 1, b);
      for (int s = 0; s < np; ++s) {
        long e = UP.rowptr[giu[i]] + nbr_pos(nbp, gp_[s]);
        for (int c = 0; c < d; ++c) UP.val[e * d + c] += Ce[s * du + i * d + c];
      }
    }
    if (disc) { // cell-private blocks: no scatter
      std::copy(Ce.begin(), Ce.end(), cellC.begin() + (size_t)c * np * du);
      double *mb = cellMB.data() + (size_t)c * np * np * 2;
      for (int i = 0; i < np * np; ++i) {
        mb[2 * i] = Mp[i];
        mb[2 * i + 1] = Be[i];
      }
      continue;
    }
    for (int s = 0; s < np; ++s) {
      NbrBox nbu = nbr_box(gp_[s], r - 1, r, b), nbp = nbr_box(gp_[s], r - 1, r - 1, b);
      for (int j = 0; j < nu; ++j) {
        long e = PU.rowptr[gip[s]] + nbr_pos(nbu, gu_[j]);
        for (int cp = 0; cp < d; ++cp) PU.val[e * d + cp] += Ce[s * du + j * d + cp];
        if (b1)
          for (int cp = 0; cp < d; ++cp) PUv.val[e * d + cp] += Cv[s * du + j * d + cp];
      }
      for (int t = 0; t < np; ++t) {
        long e = PP.rowptr[gip[s]] + nbr_pos(nbp, gp_[t]);
        PP.val[e * 2 + 0] += Mp[s * np + t];
        PP.val[e * 2 + 1] += Be[s * np + t];
      }
    }
  }
  }
  }

  // expand to the spatial system CSR (rows u-eq, v-eq, p-eq; cols V, U, P)
  const double rho = coef.rho, c0 = coef.c0;
  const long R = L.R, S = L.S, ns = L.ns;
  if (disc) {
    expand_disc(L, UU, cellC, cellMB, RU, gam_b, b1);
    if (b1) {
      // -Cvol per pressure dof over its cell's nodes (the layout of the
      // device's p-row coupling); the volume element matrix is the same on
      // every cell
      L.cvol.resize((size_t)L.S * nu * d);
      for (long sI = 0; sI < L.S; ++sI) {
        const int sl = (int)(sI % np);
        for (int j = 0; j < nu; ++j)
          for (int cp = 0; cp < d; ++cp) L.cvol[((size_t)sI * nu + j) * d + cp] = -Cv[sl * du + j * d + cp];
      }
    }
    return L;
  }
  L.rowptr.assign(ns + 1, 0);
  int a[3];
  for (long I = 0; I < L.U.nnodes; ++I) {
    long nnu = UU.rowptr[I + 1] - UU.rowptr[I], nnp = UP.rowptr[I + 1] - UP.rowptr[I];
    for (int c = 0; c < d; ++c) {
      L.rowptr[I * d + c + 1] = 2 * nnu;
      L.rowptr[R + I * d + c + 1] = nnu + d * nnu + nnp;
    }
  }
  for (long s = 0; s < S; ++s)
    L.rowptr[2 * R + s + 1] = d * (PU.rowptr[s + 1] - PU.rowptr[s]) + (PP.rowptr[s + 1] - PP.rowptr[s]);
  for (long i = 0; i < ns; ++i) L.rowptr[i + 1] += L.rowptr[i];
  const long nnz = L.rowptr[ns];
  L.col.resize(nnz);
  L.v1.resize(nnz);
  L.v2.resize(nnz);
  // rows are disjoint ranges of the CSR: threaded, and every entry of col, v1
  // and v2 is written once here (the arrays start uninitialised)
#pragma omp parallel for schedule(dynamic, 64)
  for (long I = 0; I < L.U.nnodes; ++I) {
    int a[3];
    unflatten(I, L.U.dims, d, a);
    NbrBox nbu = nbr_box(a, r, r, b), nbp = nbr_box(a, r, r - 1, b);
    std::vector<long> Jn(nbu.size), Sn(nbp.size);
    long t = 0;
    for (int z = 0; z < nbu.ext[2]; ++z)
      for (int y = 0; y < nbu.ext[1]; ++y)
        for (int x = 0; x < nbu.ext[0]; ++x) {
          int aj[3] = {nbu.lo[0] + x, nbu.lo[1] + y, nbu.lo[2] + z};
          Jn[t++] = flatten(aj, L.U.dims);
        }
    t = 0;
    for (int z = 0; z < nbp.ext[2]; ++z)
      for (int y = 0; y < nbp.ext[1]; ++y)
        for (int x = 0; x < nbp.ext[0]; ++x) {
          int aj[3] = {nbp.lo[0] + x, nbp.lo[1] + y, nbp.lo[2] + z};
          Sn[t++] = flatten(aj, L.P.dims);
        }
    const double *uu = &UU.val[UU.rowptr[I] * UU.nvals];
    const double *up = &UP.val[UP.rowptr[I] * d];
    for (int c = 0; c < d; ++c) {
      // u-equation row (multiplied by rho): -rho M on V (W), rho M on U (Dt)
      long e = L.rowptr[I * d + c];
      for (long j = 0; j < nbu.size; ++j, ++e) {
        L.col[e] = (int)(Jn[j] * d + c);
        L.v1[e] = 0.0;
        L.v2[e] = -rho * uu[j * UU.nvals];
      }
      for (long j = 0; j < nbu.size; ++j, ++e) {
        L.col[e] = (int)(R + Jn[j] * d + c);
        L.v1[e] = rho * uu[j * UU.nvals];
        L.v2[e] = 0.0;
      }
      // v-equation row: rho M on V (Dt), K on U (W), C^T on P (W)
      e = L.rowptr[R + I * d + c];
      for (long j = 0; j < nbu.size; ++j, ++e) {
        L.col[e] = (int)(Jn[j] * d + c);
        L.v1[e] = rho * uu[j * UU.nvals];
        L.v2[e] = 0.0;
      }
      for (long j = 0; j < nbu.size; ++j)
        for (int cp = 0; cp < d; ++cp, ++e) {
          L.col[e] = (int)(R + Jn[j] * d + cp);
          L.v1[e] = 0.0;
          L.v2[e] = uu[j * UU.nvals + 1 + c * d + cp];
        }
      for (long s = 0; s < nbp.size; ++s, ++e) {
        L.col[e] = (int)(2 * R + Sn[s]);
        L.v1[e] = 0.0;
        L.v2[e] = up[s * d + c];
      }
    }
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (long s = 0; s < S; ++s) {
    int a[3];
    unflatten(s, L.P.dims, d, a);
    NbrBox nbu = nbr_box(a, r - 1, r, b), nbp = nbr_box(a, r - 1, r - 1, b);
    long e = L.rowptr[2 * R + s];
    const double *pu = &PU.val[PU.rowptr[s] * d];
    const double *pp = &PP.val[PP.rowptr[s] * 2];
    long t = 0;
    for (int z = 0; z < nbu.ext[2]; ++z)
      for (int y = 0; y < nbu.ext[1]; ++y)
        for (int x = 0; x < nbu.ext[0]; ++x, ++t) {
          int aj[3] = {nbu.lo[0] + x, nbu.lo[1] + y, nbu.lo[2] + z};
          long J = flatten(aj, L.U.dims);
          for (int cp = 0; cp < d; ++cp, ++e) {
            if (b1) { // -C on U through Dt (Problem B.1)
              L.col[e] = (int)(R + J * d + cp);
              L.v1[e] = -pu[t * d + cp];
              L.v2[e] = 0.0;
            } else { // -C on V through W (Problem 3.1)
              L.col[e] = (int)(J * d + cp);
              L.v1[e] = 0.0;
              L.v2[e] = -pu[t * d + cp];
            }
          }
        }
    t = 0;
    for (int z = 0; z < nbp.ext[2]; ++z)
      for (int y = 0; y < nbp.ext[1]; ++y)
        for (int x = 0; x < nbp.ext[0]; ++x, ++t, ++e) {
          int aj[3] = {nbp.lo[0] + x, nbp.lo[1] + y, nbp.lo[2] + z};
          L.col[e] = (int)(2 * R + flatten(aj, L.P.dims));
          L.v1[e] = c0 * pp[t * 2 + 0];
          L.v2[e] = pp[t * 2 + 1];
        }
  }
  if (b1) {
    L.cvol.resize(PUv.val.size());
    for (size_t i = 0; i < PUv.val.size(); ++i) L.cvol[i] = -PUv.val[i];
  }
  return L;
}

// ---------------------------------------------------------------- transfers
CSR prolongation(const Lattice &cl, const Box &cb, const Lattice &fl, const Box &fb) {
  CSR P;
  P.nrows = fl.nnodes;
  P.ncols = cl.nnodes;
  P.rowptr.assign(P.nrows + 1, 0);
  const int m = fl.m, d = fb.dim;
  std::vector<double> v(m + 1), dd(m + 1);
  int a[3];
  for (long f = 0; f < fl.nnodes; ++f) {
    unflatten(f, fl.dims, d, a);
    double w1[3][16];
    int base[3];
    for (int i = 0; i < 3; ++i) {
      if (i < d) {
        int cf = std::min(a[i] / m, fb.n[i] - 1);
        int loc = a[i] - m * cf;
        int cc = cf / 2;
        double xi = ((cf % 2) + fl.ref[loc]) / 2.0;
        lagrange(cl.ref, xi, v.data(), dd.data());
        for (int j = 0; j <= m; ++j) w1[i][j] = v[j];
        base[i] = m * cc;
      } else {
        w1[i][0] = 1.0;
        base[i] = 0;
      }
    }
    int ez = d > 2 ? m + 1 : 1, ey = d > 1 ? m + 1 : 1;
    for (int z = 0; z < ez; ++z)
      for (int y = 0; y < ey; ++y)
        for (int x = 0; x <= m; ++x) {
          double w = w1[0][x] * w1[1][y] * w1[2][z];
          if (std::fabs(w) <= 1e-14) continue;
          int ac[3] = {base[0] + x, base[1] + y, base[2] + z};
          P.col.push_back((int)flatten(ac, cl.dims));
          P.val.push_back(w);
        }
    P.rowptr[f + 1] = (int)P.col.size();
  }
  (void)cb;
  return P;
}

int disc_basis(int m, int dim, const double *xi, int npts, std::vector<double> *phi) {
  const auto ex = disc_exponents(m, dim);
  const int nl = (int)ex.size();
  phi->assign((size_t)npts * nl, 0.0);
  for (int q = 0; q < npts; ++q) {
    double vals[3][16] = {};
    for (int i = 0; i < dim; ++i)
      for (int a = 0; a <= m; ++a) {
        double p, dp;
        legendre(a, 2.0 * xi[3 * q + i] - 1.0, &p, &dp);
        vals[i][a] = p;
      }
    for (int l = 0; l < nl; ++l) {
      double v = 1.0;
      for (int i = 0; i < dim; ++i) v *= vals[i][ex[l][i]];
      (*phi)[(size_t)q * nl + l] = v;
    }
  }
  return nl;
}

CSR prolongation_disc(int m, const Box &cb, const Box &fb) {
  // on each fine cell, the parent's basis function (a polynomial of degree m
  // there) expanded in the fine cell's orthogonal Legendre basis:
  // coef_j = <phi_i^coarse, phi_j^fine> / <phi_j^fine, phi_j^fine>, by
  // Gauss quadrature exact for the products
  const int d = fb.dim;
  const auto ex = disc_exponents(m, d);
  const int nl = (int)ex.size();
  const Rule g = gauss01(m + 2);
  const int nq = (int)g.x.size();
  CSR P;
  P.nrows = fb.ncell * nl;
  P.ncols = cb.ncell * nl;
  P.rowptr.assign(P.nrows + 1, 0);
  // 1D tables: fine Legendre values at the nodes, coarse values at the
  // matching coarse points for offset o in {0, 1}
  std::vector<double> lf((size_t)(m + 1) * nq), lc[2];
  for (int o = 0; o < 2; ++o) lc[o].resize((size_t)(m + 1) * nq);
  for (int a = 0; a <= m; ++a)
    for (int k = 0; k < nq; ++k) {
      double p, dp;
      legendre(a, 2.0 * g.x[k] - 1.0, &p, &dp);
      lf[a * nq + k] = p;
      for (int o = 0; o < 2; ++o) {
        legendre(a, 2.0 * ((o + g.x[k]) / 2.0) - 1.0, &p, &dp);
        lc[o][a * nq + k] = p;
      }
    }
  // the expansion separates by axis: coef = prod_i <Lc_{e_i}, Lf_{f_i}>_i / <Lf_{f_i}, Lf_{f_i}>_i
  auto c1 = [&](int o, int ec, int ef) {
    double num = 0.0, den = 0.0;
    for (int k = 0; k < nq; ++k) {
      num += g.w[k] * lc[o][ec * nq + k] * lf[ef * nq + k];
      den += g.w[k] * lf[ef * nq + k] * lf[ef * nq + k];
    }
    return num / den;
  };
  int cf[3], cc[3];
  for (long f = 0; f < fb.ncell; ++f) {
    unflatten(f, fb.n, d, cf);
    for (int i = 0; i < 3; ++i) cc[i] = i < d ? cf[i] / 2 : 0;
    const long ccell = flatten(cc, cb.n);
    for (int j = 0; j < nl; ++j) {
      const long row = f * nl + j;
      for (int i = 0; i < nl; ++i) {
        double w = 1.0;
        for (int ax = 0; ax < d; ++ax) w *= c1(cf[ax] - 2 * cc[ax], ex[i][ax], ex[j][ax]);
        if (std::fabs(w) <= 1e-14) continue;
        P.col.push_back((int)(ccell * nl + i));
        P.val.push_back(w);
      }
      P.rowptr[row + 1] = (int)P.col.size();
    }
  }
  return P;
}

CSR transpose(const CSR &a) {
  CSR t;
  t.nrows = a.ncols;
  t.ncols = a.nrows;
  t.rowptr.assign(t.nrows + 1, 0);
  for (int c : a.col) t.rowptr[c + 1]++;
  for (long i = 0; i < t.nrows; ++i) t.rowptr[i + 1] += t.rowptr[i];
  t.col.resize(a.col.size());
  t.val.resize(a.val.size());
  std::vector<int> pos(t.rowptr.begin(), t.rowptr.end() - 1);
  for (long r = 0; r < a.nrows; ++r)
    for (int e = a.rowptr[r]; e < a.rowptr[r + 1]; ++e) {
      int p = pos[a.col[e]]++;
      t.col[p] = (int)r;
      t.val[p] = a.val[e];
    }
  return t;
}

namespace {

// A node-level matrix in CSR form with nv values per entry.
struct NodeCSR {
  long nrows = 0;
  int nv = 1;
  std::vector<long> ptr;
  hvec<int> col;
  hvec<double> val;
};

// C = Prow^T A Pcol for a node-level matrix (rows: fine row nodes, columns:
// fine column nodes), every value slot at once; rows of C are coarse row
// nodes, sorted columns.  Threaded like the scalar product below.
NodeCSR node_rap(const NodeCSR &A, const CSR &Prow, const CSR &Pcol) {
  const int nv = A.nv;
  const long nfr = A.nrows, ncc = Pcol.ncols, ncr = Prow.ncols;
  const int nt = n_threads();
  struct Buf {
    hvec<int> col;
    hvec<double> val;
  };
  auto product = [&](long nrows, auto row_terms, std::vector<long> &ptr, hvec<int> &col, hvec<double> &val) {
    // row_terms(i, emit): calls emit(J, weight, const double *v) for the terms of row i
    std::vector<Buf> buf(nt);
    std::vector<int> who(nrows), len(nrows);
    std::vector<long> at(nrows);
    std::atomic<long> next(0);
    auto work = [&](int w) {
      std::vector<double> acc((size_t)ncc * nv, 0.0);
      std::vector<char> mark(ncc, 0);
      std::vector<int> touched;
      Buf &o = buf[w];
      for (;;) {
        const long i0 = next.fetch_add(128);
        if (i0 >= nrows) break;
        for (long i = i0; i < std::min(nrows, i0 + 128); ++i) {
          touched.clear();
          row_terms(i, [&](int J, double wgt, const double *v) {
            if (!mark[J]) {
              mark[J] = 1;
              touched.push_back(J);
              for (int k = 0; k < nv; ++k) acc[(size_t)J * nv + k] = 0.0;
            }
            for (int k = 0; k < nv; ++k) acc[(size_t)J * nv + k] += wgt * v[k];
          });
          std::sort(touched.begin(), touched.end());
          who[i] = w;
          at[i] = (long)o.col.size();
          len[i] = (int)touched.size();
          for (const int J : touched) {
            o.col.push_back(J);
            for (int k = 0; k < nv; ++k) o.val.push_back(acc[(size_t)J * nv + k]);
            mark[J] = 0;
          }
        }
      }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(work, t);
    for (auto &t : th) t.join();
    ptr.assign(nrows + 1, 0);
    for (long i = 0; i < nrows; ++i) ptr[i + 1] = ptr[i] + len[i];
    col.resize(ptr[nrows]);
    val.resize((size_t)ptr[nrows] * nv);
#pragma omp parallel for schedule(dynamic, 256)
    for (long i = 0; i < nrows; ++i) {
      const Buf &b = buf[who[i]];
      std::copy(b.col.begin() + at[i], b.col.begin() + at[i] + len[i], col.begin() + ptr[i]);
      std::copy(b.val.begin() + at[i] * nv, b.val.begin() + (at[i] + len[i]) * nv, val.begin() + ptr[i] * nv);
    }
  };
  // AP = A Pcol (rows fine, columns coarse)
  NodeCSR AP;
  AP.nrows = nfr;
  AP.nv = nv;
  product(
      nfr,
      [&](long i, auto emit) {
        for (long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
          const int j = A.col[e];
          const double *v = A.val.data() + (size_t)e * nv;
          for (int f = Pcol.rowptr[j]; f < Pcol.rowptr[j + 1]; ++f) emit(Pcol.col[f], Pcol.val[f], v);
        }
      },
      AP.ptr, AP.col, AP.val);
  // C = Prow^T AP (rows coarse)
  const CSR Rt = transpose(Prow);
  NodeCSR C;
  C.nrows = ncr;
  C.nv = nv;
  product(
      ncr,
      [&](long I, auto emit) {
        for (int e = Rt.rowptr[I]; e < Rt.rowptr[I + 1]; ++e) {
          const int i = Rt.col[e];
          const double wgt = Rt.val[e];
          for (long f = AP.ptr[i]; f < AP.ptr[i + 1]; ++f) emit(AP.col[f], wgt, AP.val.data() + (size_t)f * nv);
        }
      },
      C.ptr, C.col, C.val);
  return C;
}

// The node-level blocks of a level's spatial system (rows u-eq, v-eq, p-eq;
// columns V, U, P): rho M (from the u-rows' U columns), K (d x d, v-rows' U
// columns), C^T (v-rows' P columns), the p-rows' displacement coupling (V
// columns for Problem 3.1, U columns for B.1) and (c0 Mp, B).  False when the
// level does not have exactly this structure.
struct NodeBlocks {
  NodeCSR MM, KK, UP, PU, PP;
};

bool split_nodes(const Level &L, NodeBlocks *out) {
  const int d = L.box.dim;
  const long R = L.R, nu = R / d, S = L.S;
  const bool b1 = L.form == STFEM_FORM_PROBLEM_B_1;
  NodeBlocks &B = *out;
  auto init = [](NodeCSR &m, long n, int nv) {
    m.nrows = n;
    m.nv = nv;
    m.ptr.assign(n + 1, 0);
  };
  init(B.MM, nu, 1);
  init(B.KK, nu, d * d);
  init(B.UP, nu, d);
  init(B.PU, S, d);
  init(B.PP, S, 2);
  std::atomic<bool> ok(true);
  // counts per node row (from component 0 rows)
#pragma omp parallel for schedule(dynamic, 1024)
  for (long I = 0; I < nu; ++I) {
    long nm = 0, nk = 0, np = 0;
    for (int e = L.rowptr[I * d]; e < L.rowptr[I * d + 1]; ++e)
      if (L.col[e] >= R && L.col[e] < 2 * R && (L.col[e] - R) % d == 0) ++nm;
    for (int e = L.rowptr[R + I * d]; e < L.rowptr[R + I * d + 1]; ++e) {
      const long c = L.col[e];
      if (c >= R && c < 2 * R && (c - R) % d == 0) ++nk;
      if (c >= 2 * R) ++np;
    }
    B.MM.ptr[I + 1] = nm;
    B.KK.ptr[I + 1] = nk;
    B.UP.ptr[I + 1] = np;
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (long s = 0; s < S; ++s) {
    long nuc = 0, npp = 0;
    for (int e = L.rowptr[2 * R + s]; e < L.rowptr[2 * R + s + 1]; ++e) {
      const long c = L.col[e];
      if (c >= 2 * R) ++npp;
      else if ((b1 ? (c >= R) : (c < R)) && (c % d) == 0) ++nuc;
    }
    B.PU.ptr[s + 1] = nuc;
    B.PP.ptr[s + 1] = npp;
  }
  for (NodeCSR *m : {&B.MM, &B.KK, &B.UP, &B.PU, &B.PP}) {
    for (long i = 0; i < m->nrows; ++i) m->ptr[i + 1] += m->ptr[i];
    m->col.resize(m->ptr[m->nrows]);
    m->val.resize((size_t)m->ptr[m->nrows] * m->nv);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)m->val.size(); ++i) m->val[i] = 0.0;
  }
  // values; every row of every component must fit the node pattern of
  // component 0 (checked by position)
#pragma omp parallel for schedule(dynamic, 256)
  for (long I = 0; I < nu; ++I) {
    for (int c = 0; c < d; ++c) {
      long em = B.MM.ptr[I];
      for (int e = L.rowptr[I * d + c]; e < L.rowptr[I * d + c + 1]; ++e) {
        const long col = L.col[e];
        if (col >= R && col < 2 * R) {
          if ((col - R) % d != c || em >= B.MM.ptr[I + 1] || L.v2[e] != 0.0) { ok = false; continue; }
          if (c == 0) {
            B.MM.col[em] = (int)((col - R) / d);
            B.MM.val[em] = L.v1[e];
          } else if (B.MM.col[em] != (col - R) / d || B.MM.val[em] != L.v1[e]) {
            ok = false;
          }
          ++em;
        }
      }
      if (em != B.MM.ptr[I + 1]) ok = false; // a strict prefix of component 0's pattern
      long ek = B.KK.ptr[I], ep = B.UP.ptr[I];
      for (int e = L.rowptr[R + I * d + c]; e < L.rowptr[R + I * d + c + 1]; ++e) {
        const long col = L.col[e];
        if (col >= R && col < 2 * R) {
          const long J = (col - R) / d;
          const int cp = (int)((col - R) % d);
          if (L.v1[e] != 0.0) ok = false;
          if (cp == 0) {
            if (ek >= B.KK.ptr[I + 1]) { ok = false; continue; }
            if (c == 0) B.KK.col[ek] = (int)J;
            else if (B.KK.col[ek] != J) ok = false;
            ++ek;
          }
          if (ek == B.KK.ptr[I] || B.KK.col[ek - 1] != J) { ok = false; continue; }
          B.KK.val[(size_t)(ek - 1) * d * d + c * d + cp] = L.v2[e];
        } else if (col >= 2 * R) {
          if (ep >= B.UP.ptr[I + 1] || L.v1[e] != 0.0) { ok = false; continue; }
          if (c == 0) B.UP.col[ep] = (int)(col - 2 * R);
          else if (B.UP.col[ep] != col - 2 * R) ok = false;
          B.UP.val[(size_t)ep * d + c] = L.v2[e];
          ++ep;
        }
      }
      if (ek != B.KK.ptr[I + 1] || ep != B.UP.ptr[I + 1]) ok = false;
    }
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (long s = 0; s < S; ++s) {
    long eu = B.PU.ptr[s], ep = B.PP.ptr[s];
    for (int e = L.rowptr[2 * R + s]; e < L.rowptr[2 * R + s + 1]; ++e) {
      const long col = L.col[e];
      if (col >= 2 * R) {
        B.PP.col[ep] = (int)(col - 2 * R);
        B.PP.val[(size_t)ep * 2] = L.v1[e];
        B.PP.val[(size_t)ep * 2 + 1] = L.v2[e];
        ++ep;
      } else if (b1 ? (col >= R) : (col < R)) {
        const long rem = b1 ? col - R : col;
        const int cp = (int)(rem % d);
        if ((b1 ? L.v2[e] : L.v1[e]) != 0.0) ok = false;
        if (cp == 0) {
          if (eu >= B.PU.ptr[s + 1]) { ok = false; continue; }
          B.PU.col[eu] = (int)(rem / d);
          ++eu;
        }
        if (eu == B.PU.ptr[s] || B.PU.col[eu - 1] != rem / d) { ok = false; continue; }
        B.PU.val[(size_t)(eu - 1) * d + cp] = b1 ? L.v1[e] : L.v2[e];
      } else if (L.v1[e] != 0.0 || L.v2[e] != 0.0) {
        ok = false;
      }
    }
    if (eu != B.PU.ptr[s + 1] || ep != B.PP.ptr[s + 1]) ok = false;
  }
  // the u-rows' V columns must be -rho M and the v-rows' V columns rho M
  // (checked through their counts and values)
#pragma omp parallel for schedule(dynamic, 256)
  for (long I = 0; I < nu; ++I)
    for (int c = 0; c < d; ++c) {
      long em = B.MM.ptr[I];
      for (int e = L.rowptr[I * d + c]; e < L.rowptr[I * d + c + 1]; ++e)
        if (L.col[e] < R) {
          if (em >= B.MM.ptr[I + 1] || L.col[e] != B.MM.col[em] * d + c || L.v2[e] != -B.MM.val[em] || L.v1[e] != 0.0)
            ok = false;
          ++em;
        } else if (L.col[e] >= 2 * R && (L.v1[e] != 0.0 || L.v2[e] != 0.0)) {
          ok = false;
        }
      if (em != B.MM.ptr[I + 1]) ok = false;
      em = B.MM.ptr[I];
      for (int e = L.rowptr[R + I * d + c]; e < L.rowptr[R + I * d + c + 1]; ++e)
        if (L.col[e] < R) {
          if (em >= B.MM.ptr[I + 1] || L.col[e] != B.MM.col[em] * d + c || L.v1[e] != B.MM.val[em] || L.v2[e] != 0.0)
            ok = false;
          ++em;
        }
      if (em != B.MM.ptr[I + 1]) ok = false;
    }
  return ok;
}

// Coarse spatial CSR from its node-level blocks (the layout of the fine
// level's rows: u-rows V then U columns, v-rows V, U, P, p-rows the
// displacement coupling then P).
void join_nodes(const NodeBlocks &B, Level *L) {
  const int d = L->box.dim;
  const long R = L->R, nu = R / d, S = L->S, ns = L->ns;
  const bool b1 = L->form == STFEM_FORM_PROBLEM_B_1;
  L->rowptr.assign(ns + 1, 0);
  for (long I = 0; I < nu; ++I) {
    const long nm = B.MM.ptr[I + 1] - B.MM.ptr[I], nk = B.KK.ptr[I + 1] - B.KK.ptr[I];
    const long np = B.UP.ptr[I + 1] - B.UP.ptr[I];
    for (int c = 0; c < d; ++c) {
      L->rowptr[I * d + c + 1] = (int)(2 * nm);
      L->rowptr[R + I * d + c + 1] = (int)(nm + d * nk + np);
    }
  }
  for (long s = 0; s < S; ++s)
    L->rowptr[2 * R + s + 1] = (int)(d * (B.PU.ptr[s + 1] - B.PU.ptr[s]) + (B.PP.ptr[s + 1] - B.PP.ptr[s]));
  for (long i = 0; i < ns; ++i) L->rowptr[i + 1] += L->rowptr[i];
  const long nnz = L->rowptr[ns];
  L->col.resize(nnz);
  L->v1.resize(nnz);
  L->v2.resize(nnz);
#pragma omp parallel for schedule(dynamic, 256)
  for (long I = 0; I < nu; ++I)
    for (int c = 0; c < d; ++c) {
      long e = L->rowptr[I * d + c];
      for (long m = B.MM.ptr[I]; m < B.MM.ptr[I + 1]; ++m, ++e) {
        L->col[e] = (int)(B.MM.col[m] * d + c);
        L->v1[e] = 0.0;
        L->v2[e] = -B.MM.val[m];
      }
      for (long m = B.MM.ptr[I]; m < B.MM.ptr[I + 1]; ++m, ++e) {
        L->col[e] = (int)(R + B.MM.col[m] * d + c);
        L->v1[e] = B.MM.val[m];
        L->v2[e] = 0.0;
      }
      e = L->rowptr[R + I * d + c];
      for (long m = B.MM.ptr[I]; m < B.MM.ptr[I + 1]; ++m, ++e) {
        L->col[e] = (int)(B.MM.col[m] * d + c);
        L->v1[e] = B.MM.val[m];
        L->v2[e] = 0.0;
      }
      for (long k = B.KK.ptr[I]; k < B.KK.ptr[I + 1]; ++k)
        for (int cp = 0; cp < d; ++cp, ++e) {
          L->col[e] = (int)(R + B.KK.col[k] * d + cp);
          L->v1[e] = 0.0;
          L->v2[e] = B.KK.val[(size_t)k * d * d + c * d + cp];
        }
      for (long p = B.UP.ptr[I]; p < B.UP.ptr[I + 1]; ++p, ++e) {
        L->col[e] = (int)(2 * R + B.UP.col[p]);
        L->v1[e] = 0.0;
        L->v2[e] = B.UP.val[(size_t)p * d + c];
      }
    }
#pragma omp parallel for schedule(dynamic, 256)
  for (long s = 0; s < S; ++s) {
    long e = L->rowptr[2 * R + s];
    for (long u = B.PU.ptr[s]; u < B.PU.ptr[s + 1]; ++u)
      for (int cp = 0; cp < d; ++cp, ++e) {
        const double v = B.PU.val[(size_t)u * d + cp];
        L->col[e] = (int)((b1 ? R : 0) + B.PU.col[u] * d + cp);
        L->v1[e] = b1 ? v : 0.0;
        L->v2[e] = b1 ? 0.0 : v;
      }
    for (long p = B.PP.ptr[s]; p < B.PP.ptr[s + 1]; ++p, ++e) {
      L->col[e] = (int)(2 * R + B.PP.col[p]);
      L->v1[e] = B.PP.val[(size_t)p * 2];
      L->v2[e] = B.PP.val[(size_t)p * 2 + 1];
    }
  }
}

} // namespace

bool galerkin(const Level &F, const CSR &Pu, const CSR &Pp, Level *Cl) {
  // one product P^T A P per node-level block, with vector values (d^2 fewer
  // index operations for the elasticity block than a scalar product)
  NodeBlocks B;
  if (!split_nodes(F, &B)) return false;
  NodeBlocks C;
  C.MM = node_rap(B.MM, Pu, Pu);
  C.KK = node_rap(B.KK, Pu, Pu);
  C.UP = node_rap(B.UP, Pu, Pp);
  C.PU = node_rap(B.PU, Pp, Pu);
  C.PP = node_rap(B.PP, Pp, Pp);
  join_nodes(C, Cl);
  return true;
}

// ---------------------------------------------------------------- patches
int n_threads() {
  unsigned n = std::thread::hardware_concurrency();
  return n ? (int)n : 4;
}

static bool invert_unblocked(double *a, int n) {
  std::vector<int> piv(n);
  const bool par = false;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(a[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    double *rk = a + (size_t)k * n;
    const double inv = 1.0 / rk[k];
    rk[k] = 1.0;
    for (int j = 0; j < n; ++j) rk[j] *= inv;
#pragma omp parallel for schedule(static) if (par)
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      double *ri = a + (size_t)i * n;
      const double f = ri[k];
      if (f == 0.0) continue;
      ri[k] = 0.0;
      for (int j = 0; j < n; ++j) ri[j] -= f * rk[j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k)
      for (int i = 0; i < n; ++i) std::swap(a[(size_t)i * n + k], a[(size_t)i * n + piv[k]]);
  return true;
}

// Blocked Gauss-Jordan inverse (delayed updates) for large matrices (the
// coarse level): the same eliminations and pivots as invert_unblocked, in
// panels of PB columns.  Inside a panel the panel columns of every row are
// updated at once; the other columns of the panel's pivot rows are brought up
// to date when the row becomes the pivot; all remaining updates of a panel are
// applied at its end as one rank-PB product, threaded and register-blocked,
// so the matrix is swept once per panel instead of once per pivot.
static bool invert_blocked(double *a, int n) {
  constexpr int PB = 64;
  const bool par = n >= 2048; // threads only for the coarse level (patch workers are threads already)
  std::vector<int> piv(n);
  std::vector<double> F((size_t)n * PB), R((size_t)PB * n);
  for (int k0 = 0; k0 < n; k0 += PB) {
    const int k1 = std::min(n, k0 + PB), b = k1 - k0;
    std::fill(F.begin(), F.end(), 0.0);
    for (int k = k0; k < k1; ++k) {
      const int kk = k - k0;
      int p = k;
      double best = std::fabs(a[(size_t)k * n + k]);
      for (int i = k + 1; i < n; ++i) {
        const double v = std::fabs(a[(size_t)i * n + k]);
        if (v > best) {
          best = v;
          p = i;
        }
      }
      if (!(best > 0.0) || !std::isfinite(best)) return false;
      piv[k] = p;
      if (p != k) {
        for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
        for (int j = 0; j < PB; ++j) std::swap(F[(size_t)k * PB + j], F[(size_t)p * PB + j]);
      }
      double *rk = a + (size_t)k * n;
      // pending updates of this panel's earlier steps on row k, outside the panel
      for (int q2 = 0; q2 < kk; ++q2) {
        const double f = F[(size_t)k * PB + q2];
        if (f == 0.0) continue;
        const double *rq = a + (size_t)(k0 + q2) * n;
#pragma omp parallel for schedule(static) if (par && n >= 4096)
        for (int j = 0; j < n; ++j)
          if (j < k0 || j >= k1) rk[j] -= f * rq[j];
        F[(size_t)k * PB + q2] = 0.0;
      }
      const double inv = 1.0 / rk[k];
      rk[k] = 1.0;
      for (int j = 0; j < n; ++j) rk[j] *= inv;
      // the panel columns of every other row; the multipliers are kept
#pragma omp parallel for schedule(static) if (par)
      for (int i = 0; i < n; ++i) {
        if (i == k) continue;
        double *ri = a + (size_t)i * n;
        const double f = ri[k];
        if (f == 0.0) continue;
        F[(size_t)i * PB + kk] = f;
        ri[k] = 0.0;
        for (int j = k0; j < k1; ++j) ri[j] -= f * rk[j];
      }
    }
    // the panel's pivot rows outside the panel, as they were at their steps
    for (int q2 = 0; q2 < b; ++q2)
      std::copy(a + (size_t)(k0 + q2) * n, a + (size_t)(k0 + q2 + 1) * n, R.begin() + (size_t)q2 * n);
    // rows -= F R outside the panel: four rows per pass over a column tile
    const int nblk = (n + 3) / 4;
#pragma omp parallel for schedule(dynamic, 4) if (par)
    for (int ib = 0; ib < nblk; ++ib) {
      const int i0 = ib * 4, ni = std::min(4, n - i0);
      for (int j0 = 0; j0 < n; j0 += 512) {
        const int j1 = std::min(n, j0 + 512);
        for (int q2 = 0; q2 < b; ++q2) {
          double f[4] = {0.0, 0.0, 0.0, 0.0};
          bool any = false;
          for (int t = 0; t < ni; ++t) {
            f[t] = F[(size_t)(i0 + t) * PB + q2];
            any = any || f[t] != 0.0;
          }
          if (!any) continue;
          const double *rq = R.data() + (size_t)q2 * n;
          // the tile without the panel columns: [j0, ja) and [jb, j1)
          const int ja = std::min(j1, std::max(j0, k0)), jb = std::max(j0, std::min(j1, k1));
          if (ni == 4) {
            double *r0 = a + (size_t)i0 * n, *r1 = r0 + n, *r2 = r1 + n, *r3 = r2 + n;
            const double f0 = f[0], f1 = f[1], f2 = f[2], f3 = f[3];
            for (int j = j0; j < ja; ++j) {
              const double x = rq[j];
              r0[j] -= f0 * x;
              r1[j] -= f1 * x;
              r2[j] -= f2 * x;
              r3[j] -= f3 * x;
            }
            for (int j = jb; j < j1; ++j) {
              const double x = rq[j];
              r0[j] -= f0 * x;
              r1[j] -= f1 * x;
              r2[j] -= f2 * x;
              r3[j] -= f3 * x;
            }
          } else {
            for (int t = 0; t < ni; ++t) {
              double *ri = a + (size_t)(i0 + t) * n;
              const double ft = f[t];
              for (int j = j0; j < ja; ++j) ri[j] -= ft * rq[j];
              for (int j = jb; j < j1; ++j) ri[j] -= ft * rq[j];
            }
          }
        }
      }
    }
  }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k)
      for (int i = 0; i < n; ++i) std::swap(a[(size_t)i * n + k], a[(size_t)i * n + piv[k]]);
  return true;
}

// Patch matrices (small, one per thread) take the unblocked form; the coarse
// level (large) the blocked one.
bool invert(double *a, int n) { return n >= 512 ? invert_blocked(a, n) : invert_unblocked(a, n); }

// Gauss-Jordan inverse with partial pivoting of a complex row-major matrix
// held as separate real and imaginary parts (contiguous rows vectorise);
// the elimination updates two rows per pass over the pivot row.
static bool invert_complex(double *re, double *im, int n) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::hypot(re[(size_t)k * n + k], im[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      const double v = std::hypot(re[(size_t)i * n + k], im[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        std::swap(re[(size_t)k * n + j], re[(size_t)p * n + j]);
        std::swap(im[(size_t)k * n + j], im[(size_t)p * n + j]);
      }
    double *kr = re + (size_t)k * n, *ki = im + (size_t)k * n;
    const double dr = kr[k], di = ki[k], den = dr * dr + di * di, ir = dr / den, ii = -di / den;
    kr[k] = 1.0;
    ki[k] = 0.0;
    for (int j = 0; j < n; ++j) {
      const double x = kr[j], y = ki[j];
      kr[j] = x * ir - y * ii;
      ki[j] = x * ii + y * ir;
    }
    int rows[2], nrow = 0;
    auto eliminate = [&](int cnt) {
      if (cnt == 2) {
        double *ar = re + (size_t)rows[0] * n, *ai = im + (size_t)rows[0] * n;
        double *br = re + (size_t)rows[1] * n, *bi = im + (size_t)rows[1] * n;
        const double fr = ar[k], fi = ai[k], gr = br[k], gi = bi[k];
        ar[k] = ai[k] = br[k] = bi[k] = 0.0;
        for (int j = 0; j < n; ++j) {
          const double x = kr[j], y = ki[j];
          ar[j] -= fr * x - fi * y;
          ai[j] -= fr * y + fi * x;
          br[j] -= gr * x - gi * y;
          bi[j] -= gr * y + gi * x;
        }
      } else if (cnt == 1) {
        double *ar = re + (size_t)rows[0] * n, *ai = im + (size_t)rows[0] * n;
        const double fr = ar[k], fi = ai[k];
        ar[k] = ai[k] = 0.0;
        for (int j = 0; j < n; ++j) {
          const double x = kr[j], y = ki[j];
          ar[j] -= fr * x - fi * y;
          ai[j] -= fr * y + fi * x;
        }
      }
    };
    for (int i = 0; i < n; ++i) {
      if (i == k || (re[(size_t)i * n + k] == 0.0 && im[(size_t)i * n + k] == 0.0)) continue;
      rows[nrow++] = i;
      if (nrow == 2) {
        eliminate(2);
        nrow = 0;
      }
    }
    eliminate(nrow);
  }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k)
      for (int i = 0; i < n; ++i) {
        std::swap(re[(size_t)i * n + k], re[(size_t)i * n + piv[k]]);
        std::swap(im[(size_t)i * n + k], im[(size_t)i * n + piv[k]]);
      }
  return true;
}

// The same for a std::complex array (the small q x q matrices of time_diag).
static bool invert_complex(std::complex<double> *a, int n) {
  std::vector<double> re((size_t)n * n), im((size_t)n * n);
  for (size_t i = 0; i < (size_t)n * n; ++i) {
    re[i] = a[i].real();
    im[i] = a[i].imag();
  }
  if (!invert_complex(re.data(), im.data(), n)) return false;
  for (size_t i = 0; i < (size_t)n * n; ++i) a[i] = std::complex<double>(re[i], im[i]);
  return true;
}

bool time_diag(const Temporal &Tm, double tau, TimeDiag *out, std::string *err) {
  typedef std::complex<double> cd;
  const int q = Tm.q;
  // T = W^{-1} Dt
  std::vector<double> A(q * q);
  for (int b = 0; b < q; ++b)
    for (int a = 0; a < q; ++a) A[b * q + a] = Tm.Dt[b * q + a] / (0.5 * tau * Tm.w[b]);
  // characteristic polynomial (Faddeev-LeVerrier): p(x) = x^q + c[q-1] x^{q-1} + ... + c[0]
  std::vector<double> c(q + 1, 0.0), M(q * q, 0.0), AM(q * q);
  c[q] = 1.0;
  for (int k = 1; k <= q; ++k) {
    // M_k = A M_{k-1} + c_{q-k+1} I ; c_{q-k} = -tr(A M_k) / k
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        double sacc = 0.0;
        for (int l = 0; l < q; ++l) sacc += A[i * q + l] * M[l * q + j];
        AM[i * q + j] = sacc;
      }
    for (int i = 0; i < q * q; ++i) M[i] = AM[i];
    for (int i = 0; i < q; ++i) M[i * q + i] += c[q - k + 1];
    double tr = 0.0;
    for (int i = 0; i < q; ++i)
      for (int l = 0; l < q; ++l) tr += A[i * q + l] * M[l * q + i];
    c[q - k] = -tr / k;
  }
  // roots by Durand-Kerner (Weierstrass) iteration
  auto poly = [&](cd x) {
    cd v = 1.0;
    for (int k = q - 1; k >= 0; --k) v = v * x + c[k];
    return v;
  };
  double rad = 0.0;
  for (int k = 0; k < q; ++k) rad = std::max(rad, std::abs(c[k]));
  rad = 1.0 + rad;
  std::vector<cd> z(q);
  for (int i = 0; i < q; ++i) z[i] = std::polar(0.5 * rad, 2.0 * M_PI * i / q + 0.4);
  for (int it = 0; it < 2000; ++it) {
    double delta = 0.0;
    for (int i = 0; i < q; ++i) {
      cd den = 1.0;
      for (int j = 0; j < q; ++j)
        if (j != i) den *= (z[i] - z[j]);
      const cd dz = poly(z[i]) / den;
      z[i] -= dz;
      delta = std::max(delta, std::abs(dz) / std::max(1.0, std::abs(z[i])));
    }
    if (delta < 1e-15) break;
  }
  // classify: real slots, then one member (Im > 0) of each conjugate pair
  std::vector<cd> slots;
  int nr = 0, nc = 0;
  std::vector<bool> used(q, false);
  for (int i = 0; i < q; ++i)
    if (std::fabs(z[i].imag()) <= 1e-9 * std::max(1.0, std::abs(z[i]))) {
      slots.push_back(cd(z[i].real(), 0.0));
      used[i] = true;
      ++nr;
    }
  for (int i = 0; i < q; ++i)
    if (!used[i] && z[i].imag() > 0) {
      slots.push_back(z[i]);
      ++nc;
    }
  if (nr + 2 * nc != q) {
    *err = "time matrix eigenvalues are not real or conjugate pairs";
    return false;
  }
  // eigenvectors by inverse iteration with a perturbed shift
  std::vector<cd> Vf(q * q); // full V, columns: slots then conjugates of complex slots
  std::vector<cd> lamf(q);
  int col = 0;
  auto eigvec = [&](cd lam, std::vector<cd> &v) {
    std::vector<cd> B(q * q);
    const cd mu = lam * (1.0 + 1e-11) + cd(1e-13, 0.0);
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) B[i * q + j] = A[i * q + j] - (i == j ? mu : 0.0);
    if (!invert_complex(B.data(), q)) return false;
    v.assign(q, cd(1.0, 0.3));
    for (int it = 0; it < 3; ++it) {
      std::vector<cd> w(q, 0.0);
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) w[i] += B[i * q + j] * v[j];
      // normalise: largest component = 1
      int im = 0;
      for (int i = 1; i < q; ++i)
        if (std::abs(w[i]) > std::abs(w[im])) im = i;
      const cd s0 = w[im];
      for (int i = 0; i < q; ++i) v[i] = w[i] / s0;
    }
    return true;
  };
  for (int sidx = 0; sidx < nr + nc; ++sidx) {
    std::vector<cd> v;
    if (!eigvec(slots[sidx], v)) {
      *err = "eigenvector iteration failed";
      return false;
    }
    if (sidx < nr)
      for (auto &x : v) x = cd(x.real(), 0.0);
    for (int i = 0; i < q; ++i) Vf[i * q + col] = v[i];
    lamf[col] = slots[sidx];
    ++col;
  }
  for (int sidx = nr; sidx < nr + nc; ++sidx) {
    for (int i = 0; i < q; ++i) Vf[i * q + col] = std::conj(Vf[i * q + sidx]);
    lamf[col] = std::conj(slots[sidx]);
    ++col;
  }
  std::vector<cd> Vi(Vf);
  if (!invert_complex(Vi.data(), q)) {
    *err = "eigenvector matrix is singular";
    return false;
  }
  // check V diag(lam) V^{-1} = T
  double e = 0.0, sc = 0.0;
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      cd sacc = 0.0;
      for (int l = 0; l < q; ++l) sacc += Vf[i * q + l] * lamf[l] * Vi[l * q + j];
      e = std::max(e, std::abs(sacc - A[i * q + j]));
      sc = std::max(sc, std::fabs(A[i * q + j]));
    }
  if (e > 1e-10 * sc) {
    *err = "time matrix is not diagonalisable to working accuracy";
    return false;
  }
  TimeDiag &D = *out;
  D.q = q;
  D.nr = nr;
  D.nc = nc;
  const int ns = nr + nc;
  D.lam.resize(2 * ns);
  D.Vmat.resize(2 * q * ns);
  D.Umat.resize(2 * ns * q);
  for (int a = 0; a < ns; ++a) {
    D.lam[2 * a] = lamf[a].real();
    D.lam[2 * a + 1] = lamf[a].imag();
    for (int b = 0; b < q; ++b) {
      D.Vmat[2 * (b * ns + a)] = Vf[b * q + a].real();
      D.Vmat[2 * (b * ns + a) + 1] = Vf[b * q + a].imag();
      // U = V^{-1} W^{-1}
      const cd u = Vi[a * q + b] / (0.5 * tau * Tm.w[b]);
      D.Umat[2 * (a * q + b)] = u.real();
      D.Umat[2 * (a * q + b) + 1] = u.imag();
    }
  }
  return true;
}

static void patch_axis(int v, int m, int ncell, int *lo, int *hi) {
  int c0 = std::max(v - 1, 0), c1 = std::min(v, ncell - 1);
  int alo = m * c0, ahi = m * (c1 + 1);
  *lo = (c0 == 0) ? alo : alo + 1;
  *hi = (c1 == ncell - 1) ? ahi : ahi - 1;
}

int build_patches(const Level &L, const Temporal &T, double tau, int vec, Patches *out, std::string *err,
                  bool invert_them, const TimeDiag *td, int kind) {
  const Box &b = L.box;
  const int d = b.dim, q = T.q;
  // patch centres: lattice vertices (kind 0) or cells (kind 1), x fastest
  int vdims[3] = {1, 1, 1};
  long nv = 1;
  for (int i = 0; i < d; ++i) {
    vdims[i] = kind == 1 ? b.n[i] : b.n[i] + 1;
    nv *= vdims[i];
  }
  Patches &P = *out;
  P = Patches();
  P.npatch = nv;
  P.size.resize(nv);
  P.ld.resize(nv);
  P.dof_off.resize(nv + 1);
  P.inv_off.resize(nv + 1);
  std::vector<std::vector<int>> spatial(nv);
  int v[3];
  for (long p = 0; p < nv; ++p) {
    unflatten(p, vdims, d, v);
    int ulo[3] = {0, 0, 0}, uhi[3] = {0, 0, 0}, plo[3] = {0, 0, 0}, phi[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) {
      if (kind == 1) {
        ulo[i] = L.r * v[i];
        uhi[i] = L.r * (v[i] + 1);
        plo[i] = (L.r - 1) * v[i];
        phi[i] = (L.r - 1) * (v[i] + 1);
      } else {
        patch_axis(v[i], L.r, b.n[i], &ulo[i], &uhi[i]);
        patch_axis(v[i], L.r - 1, b.n[i], &plo[i], &phi[i]);
      }
    }
    std::vector<long> un, pn;
    for (int z = ulo[2]; z <= uhi[2]; ++z)
      for (int y = ulo[1]; y <= uhi[1]; ++y)
        for (int x = ulo[0]; x <= uhi[0]; ++x) {
          int a[3] = {x, y, z};
          un.push_back(flatten(a, L.U.dims));
        }
    if (L.pdisc) {
      // the dofs of every cell of the patch (each supported in its cell)
      int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
      for (int i = 0; i < d; ++i) {
        clo[i] = kind == 1 ? v[i] : std::max(v[i] - 1, 0);
        chi[i] = kind == 1 ? v[i] : std::min(v[i], b.n[i] - 1);
      }
      for (int z = clo[2]; z <= chi[2]; ++z)
        for (int y = clo[1]; y <= chi[1]; ++y)
          for (int x = clo[0]; x <= chi[0]; ++x) {
            int cc[3] = {x, y, z};
            const long cell = flatten(cc, b.n);
            for (int l = 0; l < L.pnloc; ++l) pn.push_back(cell * L.pnloc + l);
          }
    } else {
      for (int z = plo[2]; z <= phi[2]; ++z)
        for (int y = plo[1]; y <= phi[1]; ++y)
          for (int x = plo[0]; x <= phi[0]; ++x) {
            int a[3] = {x, y, z};
            pn.push_back(flatten(a, L.P.dims));
          }
    }
    std::vector<int> &sp = spatial[p];
    for (long I : un)
      for (int c = 0; c < d; ++c) sp.push_back((int)(I * d + c));
    for (long I : un)
      for (int c = 0; c < d; ++c) sp.push_back((int)(L.R + I * d + c));
    for (long s : pn) sp.push_back((int)(2 * L.R + s));
    P.size[p] = (int)sp.size() * q;
  }
  P.dof_off[0] = 0;
  P.inv_off[0] = 0;
  P.form = td ? 1 : 0;
  P.cs.resize(nv);
  for (long p = 0; p < nv; ++p) {
    int C = P.size[p];
    const int Cs = C / q;
    P.cs[p] = Cs;
    P.dof_off[p + 1] = P.dof_off[p] + C;
    if (td) {
      const int ldR = (Cs + 3) / 4 * 4, ldC = 2 * ((Cs + 1) / 2 * 2);
      P.ld[p] = ldR;
      P.inv_off[p + 1] = P.inv_off[p] + (long long)td->nr * Cs * ldR + (long long)td->nc * Cs * ldC;
    } else {
      P.ld[p] = (C + vec - 1) / vec * vec;
      P.inv_off[p + 1] = P.inv_off[p] + (long long)C * P.ld[p];
    }
  }
  P.dofs.resize(P.dof_off[nv]);
  if (invert_them) P.inv.assign(P.inv_off[nv], 0.0);
  for (long p = 0; p < nv; ++p) {
    const std::vector<int> &sp = spatial[p];
    long long o = P.dof_off[p];
    for (int a = 0; a < q; ++a)
      for (size_t m = 0; m < sp.size(); ++m) P.dofs[o++] = (int)(a * L.ns + sp[m]);
  }
  if (!invert_them) return 0;
  // extract and invert in parallel
  std::atomic<long> next(0);
  std::atomic<long> bad(-1);
  auto work = [&]() {
    std::vector<int> loc(L.ns, -1);
    std::vector<double> S1, S2, A, Zr, Zi;
    for (;;) {
      long p = next.fetch_add(1);
      if (p >= nv) break;
      const std::vector<int> &sp = spatial[p];
      const int Cs = (int)sp.size(), C = Cs * q;
      for (int m = 0; m < Cs; ++m) loc[sp[m]] = m;
      S1.assign((size_t)Cs * Cs, 0.0);
      S2.assign((size_t)Cs * Cs, 0.0);
      for (int m = 0; m < Cs; ++m) {
        int g = sp[m];
        for (int e = L.rowptr[g]; e < L.rowptr[g + 1]; ++e) {
          int lc = loc[L.col[e]];
          if (lc < 0) continue;
          S1[(size_t)m * Cs + lc] = L.v1[e];
          S2[(size_t)m * Cs + lc] = L.v2[e];
        }
      }
      for (int m = 0; m < Cs; ++m) loc[sp[m]] = -1;
      if (td) {
        double *dst = &P.inv[P.inv_off[p]];
        const int ldR = (Cs + 3) / 4 * 4, ldC = 2 * ((Cs + 1) / 2 * 2);
        bool ok = true;
        for (int a = 0; a < td->nr && ok; ++a) {
          const double lam = td->lam[2 * a];
          A.assign((size_t)Cs * Cs, 0.0);
          for (size_t i = 0; i < (size_t)Cs * Cs; ++i) A[i] = lam * S1[i] + S2[i];
          if (!invert(A.data(), Cs)) {
            ok = false;
            break;
          }
          for (int i = 0; i < Cs; ++i)
            for (int j = 0; j < Cs; ++j) dst[(size_t)j * ldR + i] = A[(size_t)i * Cs + j];
          dst += (size_t)Cs * ldR;
        }
        for (int a = td->nr; a < td->nr + td->nc && ok; ++a) {
          const double lr = td->lam[2 * a], li = td->lam[2 * a + 1];
          Zr.resize((size_t)Cs * Cs);
          Zi.resize((size_t)Cs * Cs);
          for (size_t i = 0; i < (size_t)Cs * Cs; ++i) {
            Zr[i] = lr * S1[i] + S2[i];
            Zi[i] = li * S1[i];
          }
          if (!invert_complex(Zr.data(), Zi.data(), Cs)) {
            ok = false;
            break;
          }
          for (int i = 0; i < Cs; ++i)
            for (int j = 0; j < Cs; ++j) {
              dst[(size_t)j * ldC + 2 * i] = Zr[(size_t)i * Cs + j];
              dst[(size_t)j * ldC + 2 * i + 1] = Zi[(size_t)i * Cs + j];
            }
          dst += (size_t)Cs * ldC;
        }
        if (!ok) bad.store(p);
        continue;
      }
      A.assign((size_t)C * C, 0.0);
      for (int bb = 0; bb < q; ++bb)
        for (int aa = 0; aa < q; ++aa) {
          const double dt = T.Dt[bb * q + aa], w = (aa == bb) ? 0.5 * tau * T.w[bb] : 0.0;
          for (int m = 0; m < Cs; ++m)
            for (int mp = 0; mp < Cs; ++mp)
              A[(size_t)(bb * Cs + m) * C + aa * Cs + mp] = dt * S1[(size_t)m * Cs + mp] + w * S2[(size_t)m * Cs + mp];
        }
      if (!invert(A.data(), C)) {
        bad.store(p);
        continue;
      }
      double *dst = &P.inv[P.inv_off[p]];
      const int ld = P.ld[p];
      for (int i = 0; i < C; ++i)
        for (int j = 0; j < C; ++j) dst[(size_t)j * ld + i] = A[(size_t)i * C + j];
    }
  };
  int nt = std::min<long>(n_threads(), nv);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(work);
  for (auto &t : th) t.join();
  if (bad.load() >= 0) {
    if (err) *err = "singular patch matrix (patch " + std::to_string(bad.load()) + ")";
    return -1;
  }
  return 0;
}

void extract_patch_blocks(const Level &L, const Patches &P, int q, long p0, long p1, hvec<double> *out,
                          std::vector<long long> *off) {
  (void)q;
  off->assign(p1 - p0 + 1, 0);
  for (long p = p0; p < p1; ++p) (*off)[p - p0 + 1] = (*off)[p - p0] + 2LL * P.cs[p] * P.cs[p];
  out->resize((size_t)off->back()); // zeroed patch by patch by the workers
  std::atomic<long> next(p0);
  auto work = [&]() {
    std::vector<int> loc(L.ns, -1);
    for (;;) {
      const long p = next.fetch_add(1);
      if (p >= p1) break;
      const int Cs = P.cs[p];
      // time node 0 of the patch dof list: the spatial indices
      const int *sp = P.dofs.data() + P.dof_off[p];
      for (int m = 0; m < Cs; ++m) loc[sp[m]] = m;
      double *S1 = out->data() + (*off)[p - p0], *S2 = S1 + (size_t)Cs * Cs;
      std::fill(S1, S1 + 2 * (size_t)Cs * Cs, 0.0);
      for (int m = 0; m < Cs; ++m) {
        const int g = sp[m];
        for (int e = L.rowptr[g]; e < L.rowptr[g + 1]; ++e) {
          const int lc = loc[L.col[e]];
          if (lc < 0) continue;
          S1[(size_t)m * Cs + lc] = L.v1[e];
          S2[(size_t)m * Cs + lc] = L.v2[e];
        }
      }
      for (int m = 0; m < Cs; ++m) loc[sp[m]] = -1;
    }
  };
  const int nt = (int)std::min<long>(n_threads(), std::max(1L, p1 - p0));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(work);
  for (auto &t : th) t.join();
}

std::vector<double> dense_slab(const Level &L, const Temporal &T, double tau) {
  const long ns = L.ns, N = ns * T.q;
  std::vector<double> A((size_t)N * N, 0.0);
  for (int bb = 0; bb < T.q; ++bb)
    for (int aa = 0; aa < T.q; ++aa) {
      const double dt = T.Dt[bb * T.q + aa], w = (aa == bb) ? 0.5 * tau * T.w[bb] : 0.0;
      for (long i = 0; i < ns; ++i)
        for (int e = L.rowptr[i]; e < L.rowptr[i + 1]; ++e)
          A[(size_t)(bb * ns + i) * N + aa * ns + L.col[e]] += dt * L.v1[e] + w * L.v2[e];
    }
  return A;
}

int build_hierarchy(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                    const stfem_bcs *bcs, double tau, std::vector<Level> *levels, std::vector<CSR> *Pu,
                    std::vector<CSR> *Pp, std::string *err) {
  if (!mesh || !deg || !mat || !bcs) {
    *err = "null argument";
    return STFEM_ERR_ARG;
  }
  const int d = mesh->dim;
  if (d != 2 && d != 3) {
    *err = "dim must be 2 or 3";
    return STFEM_ERR_ARG;
  }
  if (deg->r < 2 || deg->r > 5 || (d == 3 && deg->r > 3) || deg->k < 0 || deg->k > 4) {
    *err = "unsupported degrees (need 2 <= r <= 5 (r <= 3 in 3D), 0 <= k <= 4)";
    return STFEM_ERR_ARG;
  }
  if (mesh->n_levels < 1 || mesh->n_levels > 12 || !(tau > 0.0)) {
    *err = "invalid n_levels or tau";
    return STFEM_ERR_ARG;
  }
  if (mesh->hf_mode != STFEM_HF_MEASURE && mesh->hf_mode != STFEM_HF_LENGTH) {
    *err = "invalid hf_mode";
    return STFEM_ERR_ARG;
  }
  if (mesh->coarse_op != STFEM_COARSE_GALERKIN && mesh->coarse_op != STFEM_COARSE_REDISCRETIZE) {
    *err = "invalid coarse_op";
    return STFEM_ERR_ARG;
  }
  if (deg->form != STFEM_FORM_PROBLEM_3_1 && deg->form != STFEM_FORM_PROBLEM_B_1) {
    *err = "invalid form";
    return STFEM_ERR_ARG;
  }
  if (deg->pressure != STFEM_PRESSURE_CONTINUOUS && deg->pressure != STFEM_PRESSURE_BROKEN) {
    *err = "invalid pressure space";
    return STFEM_ERR_ARG;
  }
  for (int i = 0; i < d; ++i) {
    if (mesh->n_cells[i] < 1 || (mesh->n_cells[i] % (1 << (mesh->n_levels - 1))) != 0 ||
        !(mesh->hi[i] > mesh->lo[i])) {
      *err = "n_cells must be positive and divisible by 2^(n_levels-1), and hi > lo";
      return STFEM_ERR_ARG;
    }
  }
  const int pid = bcs->problem;
  if (pid < 0 || pid > STFEM_PROBLEM_TRACE || (pid == STFEM_PROBLEM_PULSE && d != 3) ||
      ((pid == STFEM_PROBLEM_PAPER_EOC || pid == STFEM_PROBLEM_PAPER_SUPERCONV) && d != 2)) {
    *err = "unsupported problem id for this dimension";
    return STFEM_ERR_ARG;
  }
  BCs bc;
  for (int f = 0; f < 6; ++f) {
    bc.bc_u[f] = f < 2 * d ? bcs->bc_u[f] : 0;
    bc.bc_p[f] = f < 2 * d ? bcs->bc_p[f] : 0;
    if (f < 2 * d) {
      if ((bc.bc_u[f] != 0 && bc.bc_u[f] != 1) || (bc.bc_p[f] != 0 && bc.bc_p[f] != 1)) {
        *err = "boundary condition flags must be 0 or 1";
        return STFEM_ERR_ARG;
      }
      if ((pid == STFEM_PROBLEM_PAPER_EOC || pid == STFEM_PROBLEM_PAPER_SUPERCONV) && (bc.bc_u[f] || bc.bc_p[f])) {
        *err = "the problems of Eq. 5.1 and Eq. 5.3 need Dirichlet conditions on every face";
        return STFEM_ERR_ARG;
      }
    }
  }
  const int nlev = mesh->n_levels;
  std::vector<Box> boxes(nlev);
  std::vector<Coef> coefs(nlev);
  Box fine = make_box(d, mesh->lo, mesh->hi, mesh->n_cells, mesh->hf_mode);
  Coef c;
  c.rho = mat->rho;
  c.alpha = mat->alpha;
  c.c0 = mat->c0;
  c.lam.resize(fine.ncell);
  c.mu.resize(fine.ncell);
  c.kap.resize(fine.ncell);
  for (long i = 0; i < fine.ncell; ++i) {
    c.lam[i] = mat->lambda_cell_host ? mat->lambda_cell_host[i] : mat->lambda;
    c.mu[i] = mat->mu_cell_host ? mat->mu_cell_host[i] : mat->mu;
    c.kap[i] = mat->kappa_cell_host ? mat->kappa_cell_host[i] : mat->kappa;
  }
  if (mat->K_cell_host) {
    // a symmetric positive definite tensor per cell (Sylvester's criterion)
    const int dd = d * d;
    c.K.assign(mat->K_cell_host, mat->K_cell_host + (size_t)fine.ncell * dd);
    for (long i = 0; i < fine.ncell; ++i) {
      const double *k = &c.K[(size_t)i * dd];
      double scale = 0.0, tr = 0.0;
      for (int e = 0; e < dd; ++e) scale = std::max(scale, std::fabs(k[e]));
      bool ok = std::isfinite(scale) && scale > 0.0;
      for (int a = 0; a < d && ok; ++a)
        for (int b2 = a + 1; b2 < d; ++b2) ok = ok && std::fabs(k[a * d + b2] - k[b2 * d + a]) <= 1e-12 * scale;
      const double m1 = k[0], m2 = k[0] * k[d + 1] - k[1] * k[d];
      ok = ok && m1 > 0.0 && m2 > 0.0;
      if (ok && d == 3) {
        const double m3 = k[0] * (k[4] * k[8] - k[5] * k[7]) - k[1] * (k[3] * k[8] - k[5] * k[6]) +
                          k[2] * (k[3] * k[7] - k[4] * k[6]);
        ok = m3 > 0.0;
      }
      if (!ok) {
        *err = "K_cell_host: the permeability of every cell must be a symmetric positive definite tensor";
        return STFEM_ERR_ARG;
      }
      for (int a = 0; a < d; ++a) tr += k[a * d + a];
      c.kap[i] = tr / d;
    }
  }
  boxes[nlev - 1] = fine;
  coefs[nlev - 1] = c;
  for (int l = nlev - 2; l >= 0; --l) {
    coefs[l] = coarsen(coefs[l + 1], boxes[l + 1]);
    int nc[3];
    for (int i = 0; i < 3; ++i) nc[i] = i < d ? boxes[l + 1].n[i] / 2 : 1;
    boxes[l] = make_box(d, mesh->lo, mesh->hi, nc, mesh->hf_mode);
  }
  levels->assign(nlev, Level());
  const bool galerkin_ops = mesh->coarse_op == STFEM_COARSE_GALERKIN;
  for (int l = 0; l < nlev; ++l) {
    if (galerkin_ops && l < nlev - 1) {
      // sizes only; the matrix comes from the Galerkin product below
      Level &Lv = (*levels)[l];
      Lv.box = boxes[l];
      Lv.r = deg->r;
      Lv.form = deg->form;
      Lv.coef = coefs[l];
      Lv.U = make_lattice(boxes[l], deg->r);
      if (deg->pressure == STFEM_PRESSURE_BROKEN) {
        Lv.pdisc = true;
        Lv.pnloc = (int)disc_exponents(deg->r - 1, d).size();
        Lv.P = Lattice();
        Lv.P.dim = d;
        Lv.P.m = deg->r - 1;
        Lv.P.nnodes = boxes[l].ncell * Lv.pnloc;
      } else {
        Lv.P = make_lattice(boxes[l], deg->r - 1);
      }
      Lv.R = (long)d * Lv.U.nnodes;
      Lv.S = Lv.P.nnodes;
      Lv.ns = 2 * Lv.R + Lv.S;
    } else {
      (*levels)[l] = assemble_level(boxes[l], deg->r, coefs[l], bc, deg->form, deg->pressure);
    }
  }
  Pu->assign(nlev, CSR());
  Pp->assign(nlev, CSR());
  for (int l = 1; l < nlev; ++l) {
    (*Pu)[l] = prolongation((*levels)[l - 1].U, boxes[l - 1], (*levels)[l].U, boxes[l]);
    (*Pp)[l] = deg->pressure == STFEM_PRESSURE_BROKEN
                   ? prolongation_disc(deg->r - 1, boxes[l - 1], boxes[l])
                   : prolongation((*levels)[l - 1].P, boxes[l - 1], (*levels)[l].P, boxes[l]);
  }
  if (galerkin_ops)
    for (int l = nlev - 1; l >= 1; --l)
      if (!galerkin((*levels)[l], (*Pu)[l], (*Pp)[l], &(*levels)[l - 1])) {
        *err = "level " + std::to_string(l) + " does not have the node-block structure of the spatial system";
        return STFEM_ERR_STATE;
      }
  return STFEM_OK;
}

} // namespace stfem
