// Matrix-free slab operator of the finest level (Eq. 4.7 applied cell by
// cell, without the assembled spatial matrices): on a uniform box every cell
// shares one set of unit-coefficient element matrices (mass, the lambda and
// mu parts of the elasticity form, the coupling C, the pressure stiffness
// and mass, plus the Nitsche face terms of Eqs. 3.2-3.3 for cells on a
// Dirichlet face), scaled by the cell's lambda, mu, kappa.  Two passes, both
// deterministic: k_mf_cells applies each cell's element operator to its
// local values of all q time nodes and mixes the time nodes (Dt, W), writing
// the cell's local result; k_mf_gather sums, for every slab row, the results
// of the cells holding the row's node in a fixed order.  Included by
// stfem.cu inside its anonymous namespace.
//
// The element products run on the FP32 CUDA cores (this operator serves the
// FP32 residuals of the V-cycle).  Sum factorisation is not used: at the
// degrees of the workloads (Q3 in 2D, Q2 in 3D) a cell's dense products cost
// 3.8k and 19k multiply-adds per time node, and the sum-factorised
// gradient/stress/divergence sequence would save at most about a third of
// them while the pass is bound by the shared-memory reads of the products.

constexpr int MF_CELLS = 32; // cells of a tile: one per lane
constexpr int MF_WARPS = 4;  // warps per CTA: they split the element's rows
constexpr int MF_PARTS = 4;  // CTAs per tile (each stages the tile's values)

// Element data in device memory, FP32, row-major [row][column] (u dofs
// i * d + c, p dofs s), per face f = 2 axis + side.
struct MfDev {
  int d, r, nu, np, du, q;
  int n[3];                 // cells per axis
  int udims[3], pdims[3];   // lattice sizes of Q_r and Q_{r-1}
  long R, S, ns;
  long ncell;
  int pcouple;              // 0: Problem 3.1 (-C on V through W), 1: B.1 (-C on U through Dt)
  int bc_u, bc_p;           // Dirichlet faces, bit f = 2 axis + side
  float rho, c0;
  const float *Mu, *Klam, *Kmu, *Cv, *Bv, *Mp; // volume matrices
  const float *fK;   // per face: [3][du][du] (lambda, mu and penalty parts)
  const float *fC;   // per face: [np][du]
  const float *fB;   // per face: [2][np][np] (kappa and penalty parts)
  const float *lam, *mu, *kap; // per cell
  float *scratch;              // [q][2 du + np][ncell]: per-cell results, cell fastest
};



// Lane l of every warp owns cell tile * 32 + l; the MF_PARTS x MF_WARPS
// warps of a tile (MF_PARTS CTAs) split the rows of the element.  Element
// matrices are read by all lanes at the same address (one broadcast
// transaction through the read-only cache); the tile's local values sit in
// shared memory cell-fastest, so lanes read consecutive words.  Per u-node
// row (i, c) a lane forms, for every time node, M U_a, M V_a and
// K U_b + C^T P_b (K = lam Klam + mu Kmu, plus the Nitsche face terms of a
// Dirichlet face), then the u- and v-equation results
//   e_u,b = rho (sum_a Dt[b,a] M U_a - W_b M V_b),
//   e_v,b = rho sum_a Dt[b,a] M V_a + W_b (K U_b + C^T P_b);
// per p row s: Mp P_a, B P_b and C V (3.1) or C U (B.1), then
//   e_p,b = sum_a Dt[b,a] (c0 Mp P_a [- C U_a]) + W_b (B P_b [- C V_b]).
template <int Q, int D>
__global__ void __launch_bounds__(32 * MF_WARPS) k_mf_cells(MfDev A, TimeCoef<float> tc, const float *__restrict__ x) {
  extern __shared__ __align__(16) float xs[]; // [Q][nl][32]
  constexpr int d = D;
  const int nu = A.nu, np = A.np, du = A.du, nl = 2 * du + np;
  const float *__restrict__ Mu = A.Mu, *__restrict__ Klam = A.Klam, *__restrict__ Kmu = A.Kmu;
  const float *__restrict__ Cv = A.Cv, *__restrict__ Bv = A.Bv, *__restrict__ Mp = A.Mp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long ntile = (A.ncell + MF_CELLS - 1) / MF_CELLS;
  const int part = (int)(blockIdx.x % MF_PARTS);
  const int rw = part * MF_WARPS + warp; // row set of this warp
  constexpr int NW = MF_PARTS * MF_WARPS;
  for (long tile = blockIdx.x / MF_PARTS; tile < ntile; tile += gridDim.x / MF_PARTS) {
    __syncthreads(); // the previous tile's values are no longer read
    // local values of the tile's cells: entry k of time node a at
    // xs[(a * nl + k) * 32 + cell]
    for (int e = threadIdx.x; e < Q * nl * MF_CELLS; e += blockDim.x) {
      const int cl = e % MF_CELLS, ak = e / MF_CELLS, a = ak / nl, k = ak % nl;
      const long cell = tile * MF_CELLS + cl;
      float v = 0.f;
      if (cell < A.ncell) {
        int cm[3] = {0, 0, 0};
        int t = (int)cell;
#pragma unroll
        for (int i = 0; i < D; ++i) {
          cm[i] = t % A.n[i];
          t /= A.n[i];
        }
        const bool unode = k < 2 * du;
        const int deg = unode ? A.r : A.r - 1;
        int l = unode ? (k % du) / d : k - 2 * du;
        long node = 0, stride = 1;
#pragma unroll
        for (int i = 0; i < D; ++i) {
          node += (long)(deg * cm[i] + l % (deg + 1)) * stride;
          l /= deg + 1;
          stride *= unode ? A.udims[i] : A.pdims[i];
        }
        const long g = unode ? (long)a * A.ns + (k / du) * A.R + node * d + (k % du) % d
                             : (long)a * A.ns + 2 * A.R + node;
        v = x[g];
      }
      xs[e] = v;
    }
    __syncthreads();
    const long cell = tile * MF_CELLS + lane;
    const bool live = cell < A.ncell;
    float lam = 0.f, mu = 0.f, kap = 0.f;
    int fu = 0, fp = 0;
    if (live) {
      lam = A.lam[cell];
      mu = A.mu[cell];
      kap = A.kap[cell];
      int t = (int)cell;
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        const int c = t % A.n[ax];
        t /= A.n[ax];
        if (c == 0 && (A.bc_u >> (2 * ax) & 1)) fu |= 1 << (2 * ax);
        if (c == A.n[ax] - 1 && (A.bc_u >> (2 * ax + 1) & 1)) fu |= 1 << (2 * ax + 1);
        if (c == 0 && (A.bc_p >> (2 * ax) & 1)) fp |= 1 << (2 * ax);
        if (c == A.n[ax] - 1 && (A.bc_p >> (2 * ax + 1) & 1)) fp |= 1 << (2 * ax + 1);
      }
    }
    // the tile's warps take u-node rows I = rw, rw + NW, ... and p rows
    for (int I = rw; I < du; I += NW) {
      const int i = I / d, c = I % d;
      float mU[Q], mV[Q], kU[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) mU[a] = mV[a] = kU[a] = 0.f;
      for (int j = 0; j < nu; ++j) {
        const float m = Mu[i * nu + j];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          mV[a] += m * xs[(a * nl + j * d + c) * MF_CELLS + lane];
          mU[a] += m * xs[(a * nl + du + j * d + c) * MF_CELLS + lane];
        }
      }
#pragma unroll 4
      for (int J = 0; J < du; ++J) {
        const float k = lam * Klam[I * du + J] + mu * Kmu[I * du + J];
#pragma unroll
        for (int a = 0; a < Q; ++a) kU[a] += k * xs[(a * nl + du + J) * MF_CELLS + lane];
      }
      for (int s = 0; s < np; ++s) {
        const float cv = Cv[s * du + I];
#pragma unroll
        for (int a = 0; a < Q; ++a) kU[a] += cv * xs[(a * nl + 2 * du + s) * MF_CELLS + lane];
      }
      if (fu) { // Nitsche terms of the cell's Dirichlet faces (few cells)
        for (int f = 0; f < 2 * d; ++f) {
          if (!(fu >> f & 1)) continue;
          const float *kf = A.fK + (size_t)f * 3 * du * du;
          for (int J = 0; J < du; ++J) {
            const float k = lam * kf[I * du + J] + mu * kf[du * du + I * du + J] + kf[2 * du * du + I * du + J];
#pragma unroll
            for (int a = 0; a < Q; ++a) kU[a] += k * xs[(a * nl + du + J) * MF_CELLS + lane];
          }
          const float *cf = A.fC + (size_t)f * np * du;
          for (int s = 0; s < np; ++s) {
            const float cv = cf[s * du + I];
#pragma unroll
            for (int a = 0; a < Q; ++a) kU[a] += cv * xs[(a * nl + 2 * du + s) * MF_CELLS + lane];
          }
        }
      }
      if (live) {
#pragma unroll
        for (int b = 0; b < Q; ++b) {
          float eu = -tc.W[b] * mV[b], ev = tc.W[b] * kU[b], ev1 = 0.f;
#pragma unroll
          for (int a = 0; a < Q; ++a) {
            eu += tc.Dt[b * Q + a] * mU[a];
            ev1 += tc.Dt[b * Q + a] * mV[a];
          }
          A.scratch[((size_t)b * nl + I) * A.ncell + cell] = A.rho * eu;
          A.scratch[((size_t)b * nl + du + I) * A.ncell + cell] = A.rho * ev1 + ev;
        }
      }
    }
    for (int s = (rw + du) % NW; s < np; s += NW) {
      float mP[Q], bP[Q], cx[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) mP[a] = bP[a] = cx[a] = 0.f;
      for (int t = 0; t < np; ++t) {
        const float m = Mp[s * np + t], bb = kap * Bv[s * np + t];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          const float pv = xs[(a * nl + 2 * du + t) * MF_CELLS + lane];
          mP[a] += m * pv;
          bP[a] += bb * pv;
        }
      }
      // C against V (Problem 3.1) or U (Problem B.1)
      const int src = A.pcouple ? du : 0;
#pragma unroll 4
      for (int J = 0; J < du; ++J) {
        const float cv = Cv[s * du + J];
#pragma unroll
        for (int a = 0; a < Q; ++a) cx[a] += cv * xs[(a * nl + src + J) * MF_CELLS + lane];
      }
      for (int f = 0; f < 2 * d; ++f) {
        if (fu >> f & 1) {
          const float *cf = A.fC + (size_t)f * np * du;
          for (int J = 0; J < du; ++J) {
            const float cv = cf[s * du + J];
#pragma unroll
            for (int a = 0; a < Q; ++a) cx[a] += cv * xs[(a * nl + src + J) * MF_CELLS + lane];
          }
        }
        if (fp >> f & 1) {
          const float *bf = A.fB + (size_t)f * 2 * np * np;
          for (int t = 0; t < np; ++t) {
            const float bb = kap * bf[s * np + t] + bf[np * np + s * np + t];
#pragma unroll
            for (int a = 0; a < Q; ++a) bP[a] += bb * xs[(a * nl + 2 * du + t) * MF_CELLS + lane];
          }
        }
      }
      if (live) {
#pragma unroll
        for (int b = 0; b < Q; ++b) {
          float ep = tc.W[b] * (bP[b] - (A.pcouple ? 0.f : cx[b]));
#pragma unroll
          for (int a = 0; a < Q; ++a) ep += tc.Dt[b * Q + a] * (A.c0 * mP[a] - (A.pcouple ? cx[a] : 0.f));
          A.scratch[((size_t)b * nl + 2 * du + s) * A.ncell + cell] = ep;
        }
      }
    }
  }
}

// One thread per (node, time node): every slab row of the node (2 d rows of a
// u-node, one of a p-node) sums the results of the cells holding the node,
// cells in lexicographic order; mode 1 returns rhs - A x.
template <int Q, int D>
__global__ void k_mf_gather(MfDev A, const float *__restrict__ rhs, float *__restrict__ y, int mode) {
  constexpr int d = D;
  const int du = A.du, np = A.np, nl = 2 * du + np;
  const long nun = A.R / d, nnode = nun + A.S;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)Q * nnode) return;
  const int b = (int)(gid / nnode);
  const long node = gid % nnode;
  const bool unode = node < nun;
  const int deg = unode ? A.r : A.r - 1;
  const int *dims = unode ? A.udims : A.pdims;
  int a[3] = {0, 0, 0}, clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
  int t = (int)(unode ? node : node - nun);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    a[k] = t % dims[k];
    t /= dims[k];
    const int q0 = a[k] / deg;
    if (a[k] - q0 * deg == 0) {
      clo[k] = q0 > 0 ? q0 - 1 : 0;
      chi[k] = q0 < A.n[k] - 1 ? q0 : A.n[k] - 1;
    } else {
      clo[k] = chi[k] = q0;
    }
  }
  float acc[2 * D]; // u-node: [u-eq, v-eq] x D; p-node: [0]
#pragma unroll
  for (int i = 0; i < 2 * D; ++i) acc[i] = 0.f;
  for (int cz = clo[2]; cz <= chi[2]; ++cz)
    for (int cy = clo[1]; cy <= chi[1]; ++cy)
      for (int cx = clo[0]; cx <= chi[0]; ++cx) {
        int l = a[0] - deg * cx;
        if (d > 1) l += (a[1] - deg * cy) * (deg + 1);
        if (d > 2) l += (a[2] - deg * cz) * (deg + 1) * (deg + 1);
        const long cell = cx + (long)A.n[0] * (cy + (long)A.n[1] * cz);
        const float *o = A.scratch + (size_t)b * nl * A.ncell + cell;
        if (unode) {
#pragma unroll
          for (int c = 0; c < D; ++c) {
            acc[c] += o[(size_t)(l * D + c) * A.ncell];
            acc[D + c] += o[(size_t)(du + l * D + c) * A.ncell];
          }
        } else {
          acc[0] += o[(size_t)(2 * du + l) * A.ncell];
        }
      }
  if (unode) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const long i = (long)b * A.ns + blk * A.R + node * D + c;
        y[i] = mode ? rhs[i] - acc[D * blk + c] : acc[D * blk + c];
      }
  } else {
    const long i = (long)b * A.ns + 2 * A.R + (node - nun);
    y[i] = mode ? rhs[i] - acc[0] : acc[0];
  }
}
