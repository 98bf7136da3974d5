// Host-only inspection entry points of the C ABI (include/stfem.h): they
// rebuild the setup on the CPU and return what the GPU path uploads, so that
// the setup can be checked without a GPU.
#include "fem.hpp"

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
                          const stfem_bcs *bcs, double tau, int level, long long *n_patches, long long *total,
                          long long *off, int *dofs) {
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
  if (stfem::build_patches(L[level], stfem::make_temporal(deg->k), tau, 1, &P, &err, false) < 0) {
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
