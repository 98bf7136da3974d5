// CUDA kernels of the GMRES-GMG hot path (arXiv 2303.06742, Sec. 4), sm_103a.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace stfem_dev {

constexpr int MAXQ = 5;    // at most k = 4 (five Radau nodes)
constexpr int MAXM = 32;   // FGMRES restart length bound (the Gram-Schmidt kernels block k <= 32 vectors)

template <typename T>
struct TimeCoef {
  int q;
  T Dt[MAXQ * MAXQ]; // Dt[b*q+a]
  T W[MAXQ];         // tau/2 * w_b
};

// Problem data for right-hand sides and initial values (homogeneous Dirichlet data).
struct ProbDev {
  int id, dim;
  double rho, alpha, c0;
};

// Geometry of one level for node coordinates and loads.
struct GeomDev {
  int dim, r;
  double lo[3], h[3];
  int n[3];
  int udims[3], pdims[3];
  double refU[8], refP[8]; // Gauss-Lobatto points on [0,1]
};

// Tables for loads on the finest level.
struct LoadTables {
  int nq, nlu, nlp, nqf;
  const double *qx;   // [nq][3] reference points
  const double *qw;   // [nq] weights incl. |K|
  const double *phiU; // [nq][nlu]
  const double *phiP; // [nq][nlp]
  const double *fx;   // top face [nqf][3]
  const double *fw;   // [nqf] incl. face area
  const double *fphiU;
  const double *lam, *mu, *kap; // per fine cell
  int top_neumann;
  // broken pressure space: phiP holds its basis at the load points (nlp
  // dofs per cell), and the initial pressure is the L2 projection per cell
  // with the rule (pqx, pqw) of npq points and the basis values phiPP
  int pdisc, npq;
  const double *pqx, *pqw, *phiPP;
};

struct CSRDev {
  const int *ptr, *col;
  const void *val;
};

} // namespace stfem_dev
