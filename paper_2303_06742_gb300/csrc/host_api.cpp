// Host-only inspection entry points of the C ABI (include/stfem.h): they
// rebuild the setup on the CPU and return what the GPU path uploads, so that
// the setup can be checked without a GPU.
#include "fem.hpp"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace {
thread_local std::string g_host_err;

int build(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat, const stfem_bcs *bcs,
          double tau, std::vector<stfem::Level> *L, std::vector<stfem::CSR> *Pu, std::vector<stfem::CSR> *Pp) {
  return stfem::build_hierarchy(mesh, deg, mat, bcs, tau, L, Pu, Pp, &g_host_err);
}
} // namespace

extern "C" {

const char *stfem_host_last_error(void) { return g_host_err.c_str(); }

int stfem_host_invert(int n, double *a) {
  if (n < 1 || !a) {
    g_host_err = "invalid arguments";
    return STFEM_ERR_ARG;
  }
  if (!stfem::invert(a, n)) {
    g_host_err = "zero pivot";
    return STFEM_ERR_SINGULAR_PATCH;
  }
  return STFEM_OK;
}

int stfem_host_level_matrix(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                            const stfem_bcs *bcs, double tau, int level, long long *n, long long *nnz,
                            long long *rowptr, int *col, double *val) {
  std::vector<stfem::Level> L;
  std::vector<stfem::CSR> Pu, Pp;
  int rc = build(mesh, deg, mat, bcs, tau, &L, &Pu, &Pp);
  if (rc < 0) return rc;
  if (level == -1) level = (int)L.size() - 1;
  if (level < 0 || level >= (int)L.size()) {
    g_host_err = "level out of range";
    return STFEM_ERR_ARG;
  }
  const stfem::Level &Lv = L[level];
  const stfem::Temporal T = stfem::make_temporal(deg->k);
  const int q = T.q;
  const long ns = Lv.ns;
  // row (b, i): for a in 0..q-1, every entry of spatial row i
  long long total = 0;
  for (long i = 0; i < ns; ++i) total += (long long)(Lv.rowptr[i + 1] - Lv.rowptr[i]) * q;
  total *= q;
  if (n) *n = ns * q;
  if (nnz) *nnz = total;
  if (!rowptr || !col || !val) return STFEM_OK;
  long long e = 0;
  rowptr[0] = 0;
  for (int b = 0; b < q; ++b)
    for (long i = 0; i < ns; ++i) {
      for (int a = 0; a < q; ++a) {
        const double dt = T.Dt[b * q + a], w = (a == b) ? 0.5 * tau * T.w[b] : 0.0;
        for (int k = Lv.rowptr[i]; k < Lv.rowptr[i + 1]; ++k) {
          col[e] = (int)(a * ns + Lv.col[k]);
          val[e] = dt * Lv.v1[k] + w * Lv.v2[k];
          ++e;
        }
      }
      rowptr[b * ns + i + 1] = e;
    }
  return STFEM_OK;
}

int stfem_host_patch_dofs(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                          const stfem_bcs *bcs, double tau, int level, int patch_kind, long long *n_patches,
                          long long *total, long long *off, int *dofs) {
  if (patch_kind != STFEM_PATCHES_VERTEX && patch_kind != STFEM_PATCHES_CELL) {
    g_host_err = "unknown patch kind";
    return STFEM_ERR_ARG;
  }
  std::vector<stfem::Level> L;
  std::vector<stfem::CSR> Pu, Pp;
  int rc = build(mesh, deg, mat, bcs, tau, &L, &Pu, &Pp);
  if (rc < 0) return rc;
  if (level == -1) level = (int)L.size() - 1;
  if (level < 1 || level >= (int)L.size()) {
    g_host_err = "level out of range (patches exist on levels >= 1)";
    return STFEM_ERR_ARG;
  }
  stfem::Patches P;
  std::string err;
  if (stfem::build_patches(L[level], stfem::make_temporal(deg->k), tau, 1, &P, &err, false, nullptr,
                           patch_kind) < 0) {
    g_host_err = err;
    return STFEM_ERR_SINGULAR_PATCH;
  }
  if (n_patches) *n_patches = P.npatch;
  if (total) *total = (long long)P.dofs.size();
  if (!off || !dofs) return STFEM_OK;
  for (long p = 0; p <= P.npatch; ++p) off[p] = P.dof_off[p];
  for (size_t i = 0; i < P.dofs.size(); ++i) dofs[i] = P.dofs[i];
  return STFEM_OK;
}

int stfem_host_block_apply(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                           const stfem_bcs *bcs, double tau, int level, const double *x, double *y) {
  if (!x || !y) {
    g_host_err = "null argument";
    return STFEM_ERR_ARG;
  }
  std::vector<stfem::Level> L;
  std::vector<stfem::CSR> Pu, Pp;
  int rc = build(mesh, deg, mat, bcs, tau, &L, &Pu, &Pp);
  if (rc < 0) return rc;
  if (level == -1) level = (int)L.size() - 1;
  if (level < 0 || level >= (int)L.size()) {
    g_host_err = "level out of range";
    return STFEM_ERR_ARG;
  }
  const stfem::Temporal T = stfem::make_temporal(deg->k);
  std::vector<double> W(T.q);
  for (int b = 0; b < T.q; ++b) W[b] = 0.5 * tau * T.w[b];
  return stfem::block_apply_level(L[level], T.q, T.Dt.data(), W.data(), x, y, &g_host_err);
}

int stfem_host_galerkin_check(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                              const stfem_bcs *bcs, double tau, int level, long long drop_row, int drop_last) {
  std::vector<stfem::Level> L;
  std::vector<stfem::CSR> Pu, Pp;
  int rc = build(mesh, deg, mat, bcs, tau, &L, &Pu, &Pp);
  if (rc < 0) return rc;
  if (level == -1) level = (int)L.size() - 1;
  if (level < 1 || level >= (int)L.size()) {
    g_host_err = "level out of range (levels 1 .. n_levels-1 have a coarser level)";
    return STFEM_ERR_ARG;
  }
  stfem::Level F = L[level];
  if (drop_row >= 0) {
    const long nrows = (long)F.rowptr.size() - 1;
    if (drop_row >= nrows || F.rowptr[drop_row] == F.rowptr[drop_row + 1]) {
      g_host_err = "drop_row out of range or empty";
      return STFEM_ERR_ARG;
    }
    const long e = drop_last ? F.rowptr[drop_row + 1] - 1 : F.rowptr[drop_row];
    F.col.erase(F.col.begin() + e);
    F.v1.erase(F.v1.begin() + e);
    F.v2.erase(F.v2.begin() + e);
    for (long i = drop_row + 1; i <= nrows; ++i) --F.rowptr[i];
  }
  stfem::Level C = L[level - 1];
  if (!stfem::galerkin(F, Pu[level], Pp[level], &C)) {
    g_host_err = "level " + std::to_string(level) + " does not have the node-block structure of the Galerkin product";
    return STFEM_ERR_STATE;
  }
  return STFEM_OK;
}

int stfem_host_prolongation(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat,
                            const stfem_bcs *bcs, double tau, int level, int field, long long *nrows,
                            long long *ncols, long long *nnz, long long *rowptr, int *col, double *val) {
  std::vector<stfem::Level> L;
  std::vector<stfem::CSR> Pu, Pp;
  int rc = build(mesh, deg, mat, bcs, tau, &L, &Pu, &Pp);
  if (rc < 0) return rc;
  if (level == -1) level = (int)L.size() - 1;
  if (level < 1 || level >= (int)L.size() || (field != 0 && field != 1)) {
    g_host_err = "level or field out of range";
    return STFEM_ERR_ARG;
  }
  const stfem::CSR &P = field == 0 ? Pu[level] : Pp[level];
  if (nrows) *nrows = P.nrows;
  if (ncols) *ncols = P.ncols;
  if (nnz) *nnz = (long long)P.col.size();
  if (!rowptr || !col || !val) return STFEM_OK;
  for (long i = 0; i <= P.nrows; ++i) rowptr[i] = P.rowptr[i];
  for (size_t i = 0; i < P.col.size(); ++i) {
    col[i] = P.col[i];
    val[i] = P.val[i];
  }
  return STFEM_OK;
}

// Upper estimate of a handle's device bytes from the sizes alone: every
// array stfem_setup and stfem_gmg_setup allocate, with the neighbour boxes
// and patch sizes counted exactly per node / per vertex and the largest
// possible box for the level operators.
int stfem_estimate_bytes(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_gmg_params *gmg,
                         int restart, long long *bytes) {
  if (!mesh || !deg || !gmg || !bytes || restart < 1) {
    g_host_err = "null argument";
    return STFEM_ERR_ARG;
  }
  const int d = mesh->dim, r = deg->r, q = deg->k + 1, L = mesh->n_levels;
  if ((d != 2 && d != 3) || r < 2 || q < 1 || q > 5 || L < 1) {
    g_host_err = "invalid sizes";
    return STFEM_ERR_ARG;
  }
  const bool disc = deg->pressure == STFEM_PRESSURE_BROKEN;
  int pnl = 1; // dofs per cell of P_{r-1}^disc: binomial(r - 1 + d, d)
  for (int i = 1; i <= d; ++i) pnl = pnl * (r - 1 + i) / i;
  const bool mixed = gmg->precision == STFEM_MIXED;
  int form = gmg->patch_form;
  if (form == STFEM_PATCH_AUTO) form = mixed ? STFEM_PATCH_TIME_DIAGONAL : STFEM_PATCH_DENSE;
  const double sp = mixed ? 4.0 : 8.0; // V-cycle precision
  const int vec = mixed ? 4 : 2;
  const int nr = q % 2, nc = q / 2;
  double total = 0.0;
  long nfine[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) nfine[i] = mesh->n_cells[i];
  double Nfine = 0.0, ns_fine = 0.0, ncell_fine = 1.0;
  for (int l = L - 1; l >= 0; --l) {
    long n[3] = {1, 1, 1};
    double nu = 1, np = 1, nv = 1, ncell = 1;
    for (int i = 0; i < d; ++i) {
      n[i] = nfine[i] >> (L - 1 - l);
      nu *= r * n[i] + 1;
      np *= (r - 1) * n[i] + 1;
      nv *= n[i] + 1;
      ncell *= n[i];
    }
    if (disc) np = ncell * pnl;
    const double ns = 2.0 * d * nu + np, N = q * ns;
    if (l == L - 1) {
      Nfine = N;
      ns_fine = ns;
      ncell_fine = ncell;
    }
    // node-block operator (largest boxes): FP64 always, FP32 copy in mixed mode
    const double b1 = std::pow(2 * r + 1, d), b2 = std::pow(2 * r - 1, d);
    // broken pressure: a node couples to <= 2^d cells' dofs, a dof to its
    // cell's (r+1)^d nodes and to 2d+1 cell slots
    const double mat = disc ? nu * b1 * (1 + d * d) + nu * std::pow(2.0, d) * pnl * d +
                                  np * std::pow(r + 1, d) * d + np * (2 * d + 1) * pnl * 2
                            : nu * b1 * (1 + d * d) + nu * b2 * d + np * b1 * d + np * b2 * 2;
    total += mat * 8.0 + (nu + np + 2) * 8.0 + 3.0 * N * 8.0;
    if (mixed) total += mat * 4.0 + (nu + np + 2) * 8.0 + 3.0 * N * 4.0;
    // transfers to the next coarser level (P and P^T, both precisions)
    if (l >= 1) {
      const double tr = (nu * std::pow(r + 1, d) + np * (disc ? pnl : std::pow(r, d))) * 2.0;
      total += tr * (4.0 + 8.0) + 2.0 * (nu + np + 2) * 4.0;
      if (mixed) total += tr * (4.0 + 4.0) + 2.0 * (nu + np + 2) * 4.0;
    }
    // patches (levels >= 1): exact patch sizes per vertex (or per cell)
    if (l >= 1) {
      const bool cellk = gmg->patch_kind == STFEM_PATCHES_CELL;
      auto axis_cells = [cellk](long v, long ncl) {
        if (cellk) return 1.0;
        return (double)(std::min(v, ncl - 1) - std::max(v - 1, 0L) + 1);
      };
      auto axis_nodes = [cellk](long v, long ncl, int m) {
        if (cellk) return (double)(m + 1);
        const long c0 = std::max(v - 1, 0L), c1 = std::min(v, ncl - 1);
        const long alo = m * c0, ahi = m * (c1 + 1);
        const long lo = (c0 == 0) ? alo : alo + 1, hi = (c1 == ncl - 1) ? ahi : ahi - 1;
        return (double)(hi - lo + 1);
      };
      double inv = 0.0, sumC = 0.0;
      const long e = cellk ? 0 : 1;
      long vx = n[0] + e, vy = d > 1 ? n[1] + e : 1, vz = d > 2 ? n[2] + e : 1;
      for (long z = 0; z < vz; ++z)
        for (long y = 0; y < vy; ++y)
          for (long x = 0; x < vx; ++x) {
            double u = axis_nodes(x, n[0], r), pp = disc ? axis_cells(x, n[0]) : axis_nodes(x, n[0], r - 1);
            if (d > 1) {
              u *= axis_nodes(y, n[1], r);
              pp *= disc ? axis_cells(y, n[1]) : axis_nodes(y, n[1], r - 1);
            }
            if (d > 2) {
              u *= axis_nodes(z, n[2], r);
              pp *= disc ? axis_cells(z, n[2]) : axis_nodes(z, n[2], r - 1);
            }
            if (disc) pp *= pnl;
            const double Cs = 2.0 * d * u + pp, C = q * Cs;
            sumC += C;
            if (form == STFEM_PATCH_TIME_DIAGONAL) {
              const double ldR = std::ceil(Cs / 4.0) * 4.0, ldC = 2.0 * std::ceil(Cs / 2.0) * 2.0;
              inv += nr * Cs * ldR + nc * Cs * ldC;
            } else {
              inv += C * std::ceil(C / vec) * vec;
            }
          }
      total += inv * sp + sumC * (4.0 + sp + 4.0) + nv * (4 + 4 + 8 + 8 + 4) + (N + 1) * 4.0 + N * sp;
    }
    if (l == 0) total += N * N * 8.0; // dense coarse inverse
    // Problem B.1: the fine level's volume coupling (FP64)
    if (l == L - 1 && deg->form == STFEM_FORM_PROBLEM_B_1)
      total += (disc ? np * std::pow(r + 1, d) : np * b1) * d * 8.0;
  }
  // Krylov workspace and march buffers
  const double m = restart;
  total += (m + 1) * Nfine * 8.0 + m * Nfine * (mixed ? 4.0 : 8.0) + 5.0 * Nfine * 8.0 + ns_fine * 8.0;
  total += 608.0 * 65 * 8.0 + ncell_fine * q * std::pow(r + 2, d) * 4 * 8.0;
  total += 3.0 * ncell_fine * 8.0 + 64.0 * 1024.0; // coefficients, tables, scalars
  *bytes = (long long)(total * 1.05) + (1LL << 20);
  return STFEM_OK;
}

int stfem_host_temporal(int k, double *t, double *w, double *chi, double *Dt) {
  if (k < 0 || k > 4) {
    g_host_err = "k out of range";
    return STFEM_ERR_ARG;
  }
  stfem::Temporal T = stfem::make_temporal(k);
  for (int i = 0; i < T.q; ++i) {
    if (t) t[i] = T.t[i];
    if (w) w[i] = T.w[i];
    if (chi) chi[i] = T.chi_m1[i];
  }
  if (Dt)
    for (int i = 0; i < T.q * T.q; ++i) Dt[i] = T.Dt[i];
  return STFEM_OK;
}

} // extern "C"
