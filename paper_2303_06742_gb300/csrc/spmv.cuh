// The slab operator on the device: the node-block SpMV of Eq. 4.7 and its
// double-float form for the FGMRES product.  Included by stfem.cu inside its
// anonymous namespace, after the device helpers.

// ---------------------------------------------------------------- SpMV
// y_b = sum_a Dt[b,a] S1 x_a + W_b S2 x_b (mode 0) or rhs_b - (...) (mode 1):
// the slab operator A_n = Dt (x) S1 + W (x) S2 of Eq. 4.7.
// Node-block form of the same operator.  For a displacement node I with
// neighbours J (shared cell) and pressure neighbours s:
//   u-eq_b[I,c] = sum_a Dt[b,a] (Mr U_a)[I,c] - W_b (Mr V_b)[I,c]
//   v-eq_b[I,c] = sum_a Dt[b,a] (Mr V_a)[I,c] + W_b ((K U_b)[I,c] + (Ct P_b)[I,c])
// and for a pressure node s
//   p-eq_b[s]   = sum_a Dt[b,a] (Mp0 P_a)[s] + W_b ((B P_b)[s] + (Cn V_b)[s])
// (Problem 3.1), or with Problem B.1 (pcouple = 1)
//   p-eq_b[s]   = sum_a Dt[b,a] ((Mp0 P_a)[s] + (Cn U_a)[s]) + W_b (B P_b)[s]
// with Mr = rho M (scalar), K (d x d per pair), Ct = C^T (d per pair),
// Mp0 = c0 Mp, Cn = -C (d per pair).  G lanes per node.
template <typename T>
struct NodeBlockDev {
  long nu, np;
  int r;                       // displacement degree (pressure degree r - 1)
  int pcouple;                 // 0: Cn on V through W (3.1); 1: on U through Dt (B.1)
  int pdisc, pnl;              // broken pressure space: pnl dofs per cell (see disc_* below)
  int n[3];                    // cells per axis of the level
  int udims[3], pdims[3];      // lattice sizes of Q_r and Q_{r-1}
  const int *uu_ptr, *up_ptr, *pu_ptr, *pp_ptr;
  const T *uu_m, *uu_k, *up_c, *pu_c, *pp_m, *pp_b;
};

// Neighbour box of a node: the lattice nodes (degree m_col) of all cells that
// hold the node (lattice coordinate a, degree m_row).  Every level operator
// couples exactly within this box, so neighbour addresses are computed, not
// loaded.  These index helpers also run on the host, in the CPU model of the
// product that checks the layout.
struct Box3 {
  int lo[3], ext[3];
};

__host__ __device__ __forceinline__ Box3 node_box(const int *a, int m_row, int m_col, const int *ncell, int dim) {
  Box3 b;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < dim) {
      int clo, chi;
      if (a[i] % m_row == 0) {
        clo = a[i] / m_row - 1 > 0 ? a[i] / m_row - 1 : 0;
        chi = a[i] / m_row < ncell[i] - 1 ? a[i] / m_row : ncell[i] - 1;
      } else {
        clo = chi = a[i] / m_row;
      }
      b.lo[i] = m_col * clo;
      b.ext[i] = m_col * (chi + 1) - b.lo[i] + 1;
    } else {
      b.lo[i] = 0;
      b.ext[i] = 1;
    }
  }
  return b;
}

__host__ __device__ __forceinline__ long box_node(const Box3 &b, int e, const int *dims) {
  const int ex = e % b.ext[0];
  const int t = e / b.ext[0];
  const int ey = t % b.ext[1], ez = t / b.ext[1];
  return (long)(b.lo[0] + ex) + (long)dims[0] * ((b.lo[1] + ey) + (long)dims[1] * (b.lo[2] + ez));
}

__host__ __device__ __forceinline__ void lattice_coords(long idx, const int *dims, int dim, int *a) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < dim) {
      a[i] = (int)(idx % dims[i]);
      idx /= dims[i];
    } else {
      a[i] = 0;
    }
  }
}

// Broken pressure space (P_{r-1}^disc, pnl dofs per cell, numbered cell by
// cell).  A displacement node couples to the dofs of the cells around it: a
// box of cells (x fastest) times pnl.  A pressure dof couples to the (r+1)^D
// nodes of its cell (x fastest) and to 2D+1 cell slots times pnl: its own
// cell, then the lower and upper face neighbour along each axis.
__host__ __device__ __forceinline__ Box3 disc_cell_box(const int *a, int r, const int *ncell, int dim) {
  Box3 b;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < dim) {
      int clo, chi;
      if (a[i] % r == 0) {
        clo = a[i] / r - 1 > 0 ? a[i] / r - 1 : 0;
        chi = a[i] / r < ncell[i] - 1 ? a[i] / r : ncell[i] - 1;
      } else {
        clo = chi = a[i] / r;
      }
      b.lo[i] = clo;
      b.ext[i] = chi - clo + 1;
    } else {
      b.lo[i] = 0;
      b.ext[i] = 1;
    }
  }
  return b;
}

// Cell of slot `slot` next to cell cm, or -1 past the boundary.
__host__ __device__ __forceinline__ long disc_slot_cell(const int *cm, int slot, const int *ncell, int dim) {
  int c2[3] = {cm[0], cm[1], cm[2]};
  if (slot > 0) c2[(slot - 1) / 2] += ((slot - 1) % 2) ? 1 : -1;
  for (int i = 0; i < dim; ++i)
    if (c2[i] < 0 || c2[i] >= ncell[i]) return -1;
  return (long)c2[0] + (long)ncell[0] * (c2[1] + (long)ncell[1] * c2[2]);
}

// Displacement node j (x fastest over (r+1)^dim) of cell cm.
__host__ __device__ __forceinline__ long disc_cell_node(const int *cm, int j, int r, const int *udims, int dim) {
  int aj[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) {
    aj[i] = r * cm[i] + j % (r + 1);
    j /= r + 1;
  }
  return (long)aj[0] + (long)udims[0] * (aj[1] + (long)udims[1] * aj[2]);
}

template <typename T, int Q, int D, int G, bool PD = false, int CB = 1>
__global__ void __launch_bounds__(256) k_spmv_nb(NodeBlockDev<T> A, long ns, long R, TimeCoef<T> tc,
                                                 const T *__restrict__ x, const T *__restrict__ rhs,
                                                 T *__restrict__ y, int mode, int nb, long cstride) {
  constexpr int NA = 4 * Q * D;
  // nb right-hand sides (column stride cstride), CB of them per thread: a
  // node block loaded once serves CB columns.  Consecutive CTAs take the same
  // nodes of different column groups, so the node blocks are read from DRAM
  // about once and from L2 by the other groups.  Each column's sums run in
  // the same order for every CB.
  const int ngrp = nb / CB;
  const int col = (int)(blockIdx.x % (unsigned)ngrp) * CB;
  const long gid = (long)(blockIdx.x / (unsigned)ngrp) * blockDim.x + threadIdx.x;
  x += (long)col * cstride;
  y += (long)col * cstride;
  if (rhs) rhs += (long)col * cstride;
  const long node = gid / G;
  const int lane = threadIdx.x % G;
  T acc[CB][NA];
#pragma unroll
  for (int cb = 0; cb < CB; ++cb)
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[cb][i] = T(0);
  const bool is_u = node < A.nu;
  const bool is_p = !is_u && node < A.nu + A.np;
  if (is_u) {
    // acc layout: [0] Mr U, [1] Mr V, [2] K U, [3] Ct P; each Q x D
    int a[3];
    lattice_coords(node, A.udims, D, a);
    const Box3 bu = node_box(a, A.r, A.r, A.n, D);
    const int base = A.uu_ptr[node], e1 = A.uu_ptr[node + 1];
    // two neighbours per trip: their matrix and vector loads are independent
    for (int e0 = base + lane; e0 < e1; e0 += 2 * G) {
      const bool two = e0 + G < e1;
      const int eb[2] = {e0, two ? e0 + G : e0};
      long J[2];
      T m[2], k[2][D * D];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        J[t] = box_node(bu, eb[t] - base, A.udims);
        m[t] = (t == 0 || two) ? A.uu_m[eb[t]] : T(0);
#pragma unroll
        for (int i = 0; i < D * D; ++i) k[t][i] = (t == 0 || two) ? A.uu_k[(long)eb[t] * D * D + i] : T(0);
      }
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          T v[2][D], u[2][D];
#pragma unroll
          for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int c = 0; c < D; ++c) {
              v[t][c] = x[(long)cb * cstride + (long)a * ns + J[t] * D + c];
              u[t][c] = x[(long)cb * cstride + (long)a * ns + R + J[t] * D + c];
            }
#pragma unroll
          for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int c = 0; c < D; ++c) {
              acc[cb][(0 * Q + a) * D + c] += m[t] * u[t][c];
              acc[cb][(1 * Q + a) * D + c] += m[t] * v[t][c];
              T kk = T(0);
#pragma unroll
              for (int cp = 0; cp < D; ++cp) kk += k[t][c * D + cp] * u[t][cp];
              acc[cb][(2 * Q + a) * D + c] += kk;
            }
        }
    }
    const Box3 bp = PD ? disc_cell_box(a, A.r, A.n, D) : node_box(a, A.r, A.r - 1, A.n, D);
    const int f0 = A.up_ptr[node], f1 = A.up_ptr[node + 1];
    for (int e = f0 + lane; e < f1; e += G) {
      const long sI = PD ? box_node(bp, (e - f0) / A.pnl, A.n) * A.pnl + (e - f0) % A.pnl
                         : box_node(bp, e - f0, A.pdims);
      T ct[D];
#pragma unroll
      for (int c = 0; c < D; ++c) ct[c] = A.up_c[(long)e * D + c];
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          const T pv = x[(long)cb * cstride + (long)a * ns + 2 * R + sI];
#pragma unroll
          for (int c = 0; c < D; ++c) acc[cb][(3 * Q + a) * D + c] += ct[c] * pv;
        }
    }
  } else if (PD && is_p) {
    // broken pressure dof: acc layout as below
    const long sI = node - A.nu, cell = sI / A.pnl;
    int cm[3];
    lattice_coords(cell, A.n, D, cm);
    const int e0p = A.pp_ptr[sI], e1 = A.pp_ptr[sI + 1];
    for (int e = e0p + lane; e < e1; e += G) {
      const long c2 = disc_slot_cell(cm, (e - e0p) / A.pnl, A.n, D);
      if (c2 < 0) continue;
      const long s2 = c2 * A.pnl + (e - e0p) % A.pnl;
      const T m = A.pp_m[e], bb = A.pp_b[e];
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          const T pv = x[(long)cb * cstride + (long)a * ns + 2 * R + s2];
          acc[cb][a] += m * pv;
          acc[cb][Q + a] += bb * pv;
        }
    }
    const int f0 = A.pu_ptr[sI], f1 = A.pu_ptr[sI + 1];
    const long uoff = A.pcouple ? R : 0;
    for (int e = f0 + lane; e < f1; e += G) {
      const long J = disc_cell_node(cm, e - f0, A.r, A.udims, D);
      T cn[D];
#pragma unroll
      for (int c = 0; c < D; ++c) cn[c] = A.pu_c[(long)e * D + c];
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          T t = T(0);
#pragma unroll
          for (int c = 0; c < D; ++c) t += cn[c] * x[(long)cb * cstride + (long)a * ns + uoff + J * D + c];
          acc[cb][2 * Q + a] += t;
        }
    }
  } else if (is_p) {
    // acc layout: [0..Q) Mp0 P, [Q..2Q) B P, [2Q..3Q) Cn V (Cn U with pcouple)
    const long sI = node - A.nu;
    int a[3];
    lattice_coords(sI, A.pdims, D, a);
    const Box3 bp = node_box(a, A.r - 1, A.r - 1, A.n, D);
    const int e0p = A.pp_ptr[sI], e1 = A.pp_ptr[sI + 1];
    for (int e = e0p + lane; e < e1; e += G) {
      const long s2 = box_node(bp, e - e0p, A.pdims);
      const T m = A.pp_m[e], bb = A.pp_b[e];
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          const T pv = x[(long)cb * cstride + (long)a * ns + 2 * R + s2];
          acc[cb][a] += m * pv;
          acc[cb][Q + a] += bb * pv;
        }
    }
    const Box3 bu = node_box(a, A.r - 1, A.r, A.n, D);
    const int f0 = A.pu_ptr[sI], f1 = A.pu_ptr[sI + 1];
    const long uoff = A.pcouple ? R : 0; // the V or the U block of x
    for (int e = f0 + lane; e < f1; e += G) {
      const long J = box_node(bu, e - f0, A.udims);
      T cn[D];
#pragma unroll
      for (int c = 0; c < D; ++c) cn[c] = A.pu_c[(long)e * D + c];
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          T t = T(0);
#pragma unroll
          for (int c = 0; c < D; ++c) t += cn[c] * x[(long)cb * cstride + (long)a * ns + uoff + J * D + c];
          acc[cb][2 * Q + a] += t;
        }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int cb = 0; cb < CB; ++cb)
#pragma unroll
      for (int i = 0; i < NA; ++i) acc[cb][i] += __shfl_xor_sync(0xffffffffu, acc[cb][i], o);
  }
#pragma unroll
  for (int cb = 0; cb < CB; ++cb) {
    T *__restrict__ yc = y + (long)cb * cstride;
    const T *__restrict__ rc = rhs ? rhs + (long)cb * cstride : nullptr;
    if (is_u) {
      // outputs: (eq in {u, v}) x Q x D, output o written by lane o % G
#pragma unroll
      for (int o = 0; o < 2 * Q * D; ++o) {
        if (o % G != lane) continue;
        const int eq = o / (Q * D), b = (o / D) % Q, c = o % D;
        T val = T(0);
#pragma unroll
        for (int a = 0; a < Q; ++a) val += tc.Dt[b * Q + a] * acc[cb][(eq * Q + a) * D + c];
        if (eq == 0)
          val -= tc.W[b] * acc[cb][(1 * Q + b) * D + c];
        else
          val += tc.W[b] * (acc[cb][(2 * Q + b) * D + c] + acc[cb][(3 * Q + b) * D + c]);
        const long oi = (long)b * ns + eq * R + node * D + c;
        yc[oi] = mode ? rc[oi] - val : val;
      }
    } else if (is_p) {
      const long sI = node - A.nu;
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        if (b % G != lane) continue;
        T val;
        if (A.pcouple) {
          val = tc.W[b] * acc[cb][Q + b];
#pragma unroll
          for (int a = 0; a < Q; ++a) val += tc.Dt[b * Q + a] * (acc[cb][a] + acc[cb][2 * Q + a]);
        } else {
          val = tc.W[b] * (acc[cb][Q + b] + acc[cb][2 * Q + b]);
#pragma unroll
          for (int a = 0; a < Q; ++a) val += tc.Dt[b * Q + a] * acc[cb][a];
        }
        const long oi = (long)b * ns + 2 * R + sI;
        yc[oi] = mode ? rc[oi] - val : val;
      }
    }
  }
}

// ---------------------------------------------------------------- double-float SpMV
// y = A x for an FP64 operator whose every value a is held as the float pair
// (hi, lo), hi = fl32(a), lo = fl32(a - hi) (a = hi + lo to about 2^-48),
// applied to a vector that is exactly representable in FP32 (the output of
// the FP32 V-cycle).  Products and sums run on the FP32 pipes in double-float
// arithmetic: hi * x is split exactly with an FMA, lo * x is added to the
// error term, and the running sum is kept as an unevaluated pair (hi, lo)
// updated by Knuth's TwoSum.  The relative error of a row is about
// n 2^-48 of the sum of |a_j x_j| (FP64: n 2^-53), while the FP32 pipes run
// GB300's rate for FP32, far above its FP64 rate.  The Q time-node mixing
// of Eq. 4.7 at the end is FP64.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ void df_madd(DF &acc, float2 a, float x) {
  const float p = a.x * x;
  float e = fmaf(a.x, x, -p); // exact: a.x * x = p + e
  e = fmaf(a.y, x, e);
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  const float err = (acc.hi - (s - bb)) + (p - bb);
  acc.hi = s;
  acc.lo += err + e;
}

__device__ __forceinline__ void df_add(DF &acc, float bh, float bl) {
  const float s = acc.hi + bh;
  const float bb = s - acc.hi;
  const float err = (acc.hi - (s - bb)) + (bh - bb);
  acc.hi = s;
  acc.lo += err + bl;
}

__device__ __forceinline__ double df_val(const DF &a) { return (double)a.hi + (double)a.lo; }

// acc += c * a for a float-pair coefficient c and a double-float value a
__device__ __forceinline__ void df_fma(DF &acc, float2 c, const DF &a) {
  const float p = c.x * a.hi;
  float e = fmaf(c.x, a.hi, -p);
  e = fmaf(c.x, a.lo, e);
  e = fmaf(c.y, a.hi, e);
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  const float err = (acc.hi - (s - bb)) + (p - bb);
  acc.hi = s;
  acc.lo += err + e;
}

// Dt and W of Eq. 4.7 as float pairs (for the double-float time mixing)
struct TimeCoefDF {
  int q;
  float2 Dt[MAXQ * MAXQ], W[MAXQ], mW[MAXQ];
};

template <int Q, int D, int G, bool PD = false>
__global__ void __launch_bounds__(256) k_spmv_df(NodeBlockDev<float2> A, long ns, long R, TimeCoefDF tc,
                                                 const float *__restrict__ x, double *__restrict__ y, int nb,
                                                 long cstride) {
  constexpr int NA = 4 * Q * D;
  const int col = (int)(blockIdx.x % (unsigned)nb);
  const long gid = (long)(blockIdx.x / (unsigned)nb) * blockDim.x + threadIdx.x;
  x += (long)col * cstride;
  y += (long)col * cstride;
  const long node = gid / G;
  const int lane = threadIdx.x % G;
  DF acc[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) acc[i] = DF{0.f, 0.f};
  const bool is_u = node < A.nu;
  const bool is_p = !is_u && node < A.nu + A.np;
  if (is_u) {
    // acc layout as in k_spmv_nb: [0] M U, [1] M V, [2] K U, [3] Ct P
    int a[3];
    lattice_coords(node, A.udims, D, a);
    const Box3 bu = node_box(a, A.r, A.r, A.n, D);
    const int base = A.uu_ptr[node], e1 = A.uu_ptr[node + 1];
    for (int e = base + lane; e < e1; e += G) {
      const long J = box_node(bu, e - base, A.udims);
      const float2 m = A.uu_m[e];
      float2 k[D * D];
#pragma unroll
      for (int i = 0; i < D * D; ++i) k[i] = A.uu_k[(long)e * D * D + i];
#pragma unroll
      for (int t = 0; t < Q; ++t) {
        float v[D], u[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          v[c] = x[(long)t * ns + J * D + c];
          u[c] = x[(long)t * ns + R + J * D + c];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
          df_madd(acc[(0 * Q + t) * D + c], m, u[c]);
          df_madd(acc[(1 * Q + t) * D + c], m, v[c]);
#pragma unroll
          for (int cp = 0; cp < D; ++cp) df_madd(acc[(2 * Q + t) * D + c], k[c * D + cp], u[cp]);
        }
      }
    }
    const Box3 bp = PD ? disc_cell_box(a, A.r, A.n, D) : node_box(a, A.r, A.r - 1, A.n, D);
    const int f0 = A.up_ptr[node], f1 = A.up_ptr[node + 1];
    for (int e = f0 + lane; e < f1; e += G) {
      const long sI = PD ? box_node(bp, (e - f0) / A.pnl, A.n) * A.pnl + (e - f0) % A.pnl
                         : box_node(bp, e - f0, A.pdims);
      float2 ct[D];
#pragma unroll
      for (int c = 0; c < D; ++c) ct[c] = A.up_c[(long)e * D + c];
#pragma unroll
      for (int t = 0; t < Q; ++t) {
        const float pv = x[(long)t * ns + 2 * R + sI];
#pragma unroll
        for (int c = 0; c < D; ++c) df_madd(acc[(3 * Q + t) * D + c], ct[c], pv);
      }
    }
  } else if (PD && is_p) {
    // broken pressure dof (see k_spmv_nb)
    const long sI = node - A.nu, cell = sI / A.pnl;
    int cm[3];
    lattice_coords(cell, A.n, D, cm);
    const int e0p = A.pp_ptr[sI], e1 = A.pp_ptr[sI + 1];
    for (int e = e0p + lane; e < e1; e += G) {
      const long c2 = disc_slot_cell(cm, (e - e0p) / A.pnl, A.n, D);
      if (c2 < 0) continue;
      const long s2 = c2 * A.pnl + (e - e0p) % A.pnl;
      const float2 m = A.pp_m[e], bb = A.pp_b[e];
#pragma unroll
      for (int t = 0; t < Q; ++t) {
        const float pv = x[(long)t * ns + 2 * R + s2];
        df_madd(acc[t], m, pv);
        df_madd(acc[Q + t], bb, pv);
      }
    }
    const int f0 = A.pu_ptr[sI], f1 = A.pu_ptr[sI + 1];
    const long uoff = A.pcouple ? R : 0;
    for (int e = f0 + lane; e < f1; e += G) {
      const long J = disc_cell_node(cm, e - f0, A.r, A.udims, D);
      float2 cn[D];
#pragma unroll
      for (int c = 0; c < D; ++c) cn[c] = A.pu_c[(long)e * D + c];
#pragma unroll
      for (int t = 0; t < Q; ++t)
#pragma unroll
        for (int c = 0; c < D; ++c) df_madd(acc[2 * Q + t], cn[c], x[(long)t * ns + uoff + J * D + c]);
    }
  } else if (is_p) {
    // acc layout: [0..Q) Mp0 P, [Q..2Q) B P, [2Q..3Q) Cn V (Cn U with pcouple)
    const long sI = node - A.nu;
    int a[3];
    lattice_coords(sI, A.pdims, D, a);
    const Box3 bp = node_box(a, A.r - 1, A.r - 1, A.n, D);
    const int e0p = A.pp_ptr[sI], e1 = A.pp_ptr[sI + 1];
    for (int e = e0p + lane; e < e1; e += G) {
      const long s2 = box_node(bp, e - e0p, A.pdims);
      const float2 m = A.pp_m[e], bb = A.pp_b[e];
#pragma unroll
      for (int t = 0; t < Q; ++t) {
        const float pv = x[(long)t * ns + 2 * R + s2];
        df_madd(acc[t], m, pv);
        df_madd(acc[Q + t], bb, pv);
      }
    }
    const Box3 bu = node_box(a, A.r - 1, A.r, A.n, D);
    const int f0 = A.pu_ptr[sI], f1 = A.pu_ptr[sI + 1];
    const long uoff = A.pcouple ? R : 0; // the V or the U block of x
    for (int e = f0 + lane; e < f1; e += G) {
      const long J = box_node(bu, e - f0, A.udims);
      float2 cn[D];
#pragma unroll
      for (int c = 0; c < D; ++c) cn[c] = A.pu_c[(long)e * D + c];
#pragma unroll
      for (int t = 0; t < Q; ++t)
#pragma unroll
        for (int c = 0; c < D; ++c) df_madd(acc[2 * Q + t], cn[c], x[(long)t * ns + uoff + J * D + c]);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const float bh = __shfl_xor_sync(0xffffffffu, acc[i].hi, o);
      const float bl = __shfl_xor_sync(0xffffffffu, acc[i].lo, o);
      df_add(acc[i], bh, bl);
    }
  }
  // time-node mixing of Eq. 4.7 in double-float as well; one conversion to
  // FP64 per output
  if (is_u) {
#pragma unroll
    for (int o = 0; o < 2 * Q * D; ++o) {
      if (o % G != lane) continue;
      const int eq = o / (Q * D), b = (o / D) % Q, c = o % D;
      DF val{0.f, 0.f};
#pragma unroll
      for (int t = 0; t < Q; ++t) df_fma(val, tc.Dt[b * Q + t], acc[(eq * Q + t) * D + c]);
      if (eq == 0) {
        df_fma(val, tc.mW[b], acc[(1 * Q + b) * D + c]);
      } else {
        df_fma(val, tc.W[b], acc[(2 * Q + b) * D + c]);
        df_fma(val, tc.W[b], acc[(3 * Q + b) * D + c]);
      }
      y[(long)b * ns + eq * R + node * D + c] = df_val(val);
    }
  } else if (is_p) {
    const long sI = node - A.nu;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      if (b % G != lane) continue;
      DF val{0.f, 0.f};
      df_fma(val, tc.W[b], acc[Q + b]);
      if (!A.pcouple) df_fma(val, tc.W[b], acc[2 * Q + b]);
#pragma unroll
      for (int t = 0; t < Q; ++t) df_fma(val, tc.Dt[b * Q + t], acc[t]);
      if (A.pcouple)
#pragma unroll
        for (int t = 0; t < Q; ++t) df_fma(val, tc.Dt[b * Q + t], acc[2 * Q + t]);
      y[(long)b * ns + 2 * R + sI] = df_val(val);
    }
  }
}
