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

// Problem data for right-hand sides and initial values.  data = 1: the
// boundary data terms of Eq. 3.4 are nonzero (k_rhs_data runs); b1: Problem
// B.1's previous-slab coupling; bc_u / bc_p: 0 Dirichlet, 1 Neumann per face
// f = 2 axis + side; hF and the Nitsche penalties gam_a, gam_b of Sec. 3.
struct ProbDev {
  int id, dim;
  double rho, alpha, c0;
  int data, b1;
  int bc_u[6], bc_p[6];
  double hF, gam_a, gam_b;
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
  const double *lam, *mu; // per fine cell
  const double *Kt;       // permeability per fine cell, 3 x 3 row-major (zero-padded in 2D)
  int top_neumann;
  // broken pressure space: phiP holds its basis at the load points (nlp
  // dofs per cell), and the initial pressure is the L2 projection per cell
  // with the rule (pqx, pqw) of npq points and the basis values phiPP
  int pdisc, npq;
  const double *pqx, *pqw, *phiPP;
  // face rule of the boundary data terms, face-major (f = 2 axis + side):
  // nqd points per face, reference points dfx [f][nqd][3], weights dfw
  // [f][nqd] incl. the face measure, displacement basis dfU [f][nqd][nlu] and
  // physical gradients dfdU [f][nqd][nlu][dim], pressure basis dfP / dfdP
  int nqd;
  const double *dfx, *dfw, *dfU, *dfdU, *dfP, *dfdP;
};

struct CSRDev {
  const int *ptr, *col;
  const void *val;
};

} // namespace stfem_dev
