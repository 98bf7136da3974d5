// Patch apply of the Vanka smoother (Algorithm 4.1) for the dense and the
// time-diagonal inverses, and the averaged update d += omega D^{-1} sum.
// Included by stfem.cu inside its anonymous namespace, after the device
// helpers.

// ---------------------------------------------------------------- Vanka
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <typename T>
__device__ __forceinline__ void fma_vec(T *acc, const typename Vec16<T>::type &a, T r);
template <>
__device__ __forceinline__ void fma_vec<float>(float *acc, const float4 &a, float r) {
  acc[0] += a.x * r;
  acc[1] += a.y * r;
  acc[2] += a.z * r;
  acc[3] += a.w * r;
}
template <>
__device__ __forceinline__ void fma_vec<double>(double *acc, const double2 &a, double r) {
  acc[0] += a.x * r;
  acc[1] += a.y * r;
}

// y_P = A_P^{-1} R_P res for every patch P of the level (one CTA per patch).
// The inverse is column-major with leading dimension ld_P (multiple of VEC);
// thread (tr, tj) owns VEC consecutive rows starting at VEC*tr and the
// columns j = tj, tj + J, ...: each warp streams 32 x 16 contiguous bytes per
// column.  With J > 1 (levels with few patches) the J partial sums are added
// in a fixed order through shared memory, so the result is deterministic.
template <typename T, int J>
__global__ void __launch_bounds__(1024) k_patch_apply(const int *__restrict__ psize,
                                                      const long long *__restrict__ pdoff,
                                                      const int *__restrict__ pdofs,
                                                      const long long *__restrict__ pioff,
                                                      const int *__restrict__ pld, const T *__restrict__ pinv,
                                                      const T *__restrict__ res, T *__restrict__ y) {
  using V = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RT = blockDim.x / J;
  const int tr = threadIdx.x % RT, tj = threadIdx.x / RT;
  const long p = blockIdx.x;
  const int C = psize[p];
  const long long doff = pdoff[p];
  T *red = reinterpret_cast<T *>(smem_raw);             // [J][RT][VEC]
  T *rs = red + (J > 1 ? (size_t)J * RT * VEC : 0);     // [C]
  for (int j = threadIdx.x; j < C; j += blockDim.x) rs[j] = res[pdofs[doff + j]];
  __syncthreads();
  const T *A = pinv + pioff[p];
  const long stride = pld[p] / VEC;
  for (int base = 0; base < C; base += VEC * RT) {
    const int row0 = base + VEC * tr;
    T acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = T(0);
    if (row0 < C) {
      const V *col0 = reinterpret_cast<const V *>(A + row0);
      int j = tj;
      for (; j + 7 * J < C; j += 8 * J) {
        V a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = __ldcs(col0 + (long)(j + u * J) * stride);
#pragma unroll
        for (int u = 0; u < 8; ++u) fma_vec<T>(acc, a[u], rs[j + u * J]);
      }
      for (; j < C; j += J) fma_vec<T>(acc, __ldcs(col0 + (long)j * stride), rs[j]);
    }
    if (J > 1) {
#pragma unroll
      for (int v = 0; v < VEC; ++v) red[((size_t)tj * RT + tr) * VEC + v] = acc[v];
      __syncthreads();
      if (tj == 0 && row0 < C) {
        for (int t = 1; t < J; ++t)
#pragma unroll
          for (int v = 0; v < VEC; ++v) acc[v] += red[((size_t)t * RT + tr) * VEC + v];
#pragma unroll
        for (int v = 0; v < VEC; ++v)
          if (row0 + v < C) y[doff + row0 + v] = acc[v];
      }
      __syncthreads();
    } else if (row0 < C) {
#pragma unroll
      for (int v = 0; v < VEC; ++v)
        if (row0 + v < C) y[doff + row0 + v] = acc[v];
    }
  }
}

// Time-diagonal form of the same product.  With W^{-1} Dt = V diag(lam) V^{-1}
// (q x q) the patch matrix Dt (x) S1_P + W (x) S2_P has the inverse
//   A_P^{-1} = (V (x) I) blockdiag_a (lam_a S1_P + S2_P)^{-1} (V^{-1} W^{-1} (x) I),
// and a complex-conjugate pair of eigenvalues shares one complex block.  Per
// patch the kernel (1) gathers r_P, (2) mixes the q time blocks with
// U = V^{-1} W^{-1}, (3) multiplies each slot by its stored inverse (real
// slots: VEC rows per thread; complex slots: VEC/2 rows, (re, im) interleaved),
// (4) mixes back with V (a conjugate pair contributes 2 Re(V z)).
template <typename T>
struct DiagCoef {
  int nr, nc;
  T U[2 * MAXQ * MAXQ]; // U[(a * q + b) * 2 + {re, im}] for the slots a
  T V[2 * MAXQ * MAXQ]; // V[(b * ns + a) * 2 + {re, im}]
};

template <typename T, int J, int Q>
__global__ void __launch_bounds__(1024) k_patch_apply_diag(const int *__restrict__ pcs,
                                                           const long long *__restrict__ pdoff,
                                                           const int *__restrict__ pdofs,
                                                           const long long *__restrict__ pioff,
                                                           const T *__restrict__ pinv, const T *__restrict__ res,
                                                           T *__restrict__ y, DiagCoef<T> dc, int maxCs) {
  using Vv = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  constexpr int CR = VEC / 2; // complex rows per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RT = blockDim.x / J;
  const int tr = threadIdx.x % RT, tj = threadIdx.x / RT;
  const long p = blockIdx.x;
  const int Cs = pcs[p], C = Q * Cs;
  const long long doff = pdoff[p];
  const int nr = dc.nr, nc = dc.nc, ns = nr + nc, nrow = nr + 2 * nc;
  T *red = reinterpret_cast<T *>(smem_raw);
  T *rs = red + (J > 1 ? (size_t)J * RT * VEC : 0);
  T *rt = rs + (size_t)Q * maxCs;
  T *z = rt + (size_t)nrow * maxCs;
  for (int j = threadIdx.x; j < C; j += blockDim.x) rs[j] = res[pdofs[doff + j]];
  __syncthreads();
  for (int m = threadIdx.x; m < Cs; m += blockDim.x) {
    for (int a = 0; a < ns; ++a) {
      T re = T(0), im = T(0);
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        const T r = rs[b * Cs + m];
        re += dc.U[(a * Q + b) * 2] * r;
        im += dc.U[(a * Q + b) * 2 + 1] * r;
      }
      if (a < nr) {
        rt[a * Cs + m] = re;
      } else {
        rt[(nr + 2 * (a - nr)) * Cs + m] = re;
        rt[(nr + 2 * (a - nr) + 1) * Cs + m] = im;
      }
    }
  }
  __syncthreads();
  const int nRr = (Cs + VEC - 1) / VEC, nCr = (Cs + CR - 1) / CR;
  const int ldR = (Cs + 3) / 4 * 4, ldC = 2 * ((Cs + 1) / 2 * 2);
  const T *Ab = pinv + pioff[p];
  T vals[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) vals[v] = T(0);
  int role = -1, slot = 0, m0 = 0;
  if (tr < nr * nRr) {
    role = 0;
    slot = tr / nRr;
    m0 = VEC * (tr % nRr);
    const Vv *col0 = reinterpret_cast<const Vv *>(Ab + (size_t)slot * Cs * ldR + m0);
    const T *x = rt + slot * Cs;
    const long stride = ldR / VEC;
    int j = tj;
    for (; j + 7 * J < Cs; j += 8 * J) {
      Vv a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ldcs(col0 + (long)(j + u * J) * stride);
#pragma unroll
      for (int u = 0; u < 8; ++u) fma_vec<T>(vals, a[u], x[j + u * J]);
    }
    for (; j < Cs; j += J) fma_vec<T>(vals, __ldcs(col0 + (long)j * stride), x[j]);
  } else if (tr < nr * nRr + nc * nCr) {
    role = 1;
    const int t2 = tr - nr * nRr;
    slot = t2 / nCr;
    m0 = CR * (t2 % nCr);
    const T *A = Ab + (size_t)nr * Cs * ldR + (size_t)slot * Cs * ldC + 2 * m0;
    const T *xr = rt + (nr + 2 * slot) * Cs, *xi = xr + Cs;
    const long stride = ldC / VEC;
    const Vv *col0 = reinterpret_cast<const Vv *>(A);
    int j = tj;
    for (; STFEM_DIAG_UNROLL_COMPLEX && j + 7 * J < Cs; j += 8 * J) {
      Vv a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ldcs(col0 + (long)(j + u * J) * stride);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T *av = reinterpret_cast<const T *>(&a[u]);
        const T ar = xr[j + u * J], ai = xi[j + u * J];
#pragma unroll
        for (int i = 0; i < CR; ++i) {
          vals[2 * i] += av[2 * i] * ar - av[2 * i + 1] * ai;
          vals[2 * i + 1] += av[2 * i] * ai + av[2 * i + 1] * ar;
        }
      }
    }
    for (; j < Cs; j += J) {
      const Vv a = __ldcs(col0 + (long)j * stride);
      const T *av = reinterpret_cast<const T *>(&a);
      const T ar = xr[j], ai = xi[j];
#pragma unroll
      for (int i = 0; i < CR; ++i) {
        vals[2 * i] += av[2 * i] * ar - av[2 * i + 1] * ai;
        vals[2 * i + 1] += av[2 * i] * ai + av[2 * i + 1] * ar;
      }
    }
  }
  if (J > 1) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) red[((size_t)tj * RT + tr) * VEC + v] = vals[v];
    __syncthreads();
    if (tj == 0)
      for (int t = 1; t < J; ++t)
#pragma unroll
        for (int v = 0; v < VEC; ++v) vals[v] += red[((size_t)t * RT + tr) * VEC + v];
  }
  if (tj == 0) {
    if (role == 0) {
#pragma unroll
      for (int v = 0; v < VEC; ++v)
        if (m0 + v < Cs) z[slot * Cs + m0 + v] = vals[v];
    } else if (role == 1) {
#pragma unroll
      for (int i = 0; i < CR; ++i)
        if (m0 + i < Cs) {
          z[(nr + 2 * slot) * Cs + m0 + i] = vals[2 * i];
          z[(nr + 2 * slot + 1) * Cs + m0 + i] = vals[2 * i + 1];
        }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < C; idx += blockDim.x) {
    const int b = idx / Cs, m = idx - b * Cs;
    T val = T(0);
    for (int a = 0; a < nr; ++a) val += dc.V[(b * ns + a) * 2] * z[a * Cs + m];
    for (int c = 0; c < nc; ++c) {
      const int a = nr + c;
      val += T(2) * (dc.V[(b * ns + a) * 2] * z[(nr + 2 * c) * Cs + m] -
                     dc.V[(b * ns + a) * 2 + 1] * z[(nr + 2 * c + 1) * Cs + m]);
    }
    y[doff + idx] = val;
  }
}

// Time-diagonal patch apply for levels with few patches (latency-bound under
// the streaming kernel, whose CTAs each walk one patch's inverse chunk by
// chunk): one CTA per (patch, slot), whose threads split the slot's Cs
// columns into G groups, so that every 16-byte word of the slot's inverse is
// requested in one wave of independent loads.  Thread t owns row group
// t % nrg (VEC rows of a real slot, VEC/2 complex rows) and the columns
// t / nrg, t / nrg + G, ...; the G partial sums of a row group are added in
// the order of the groups.  The slot's result z_a goes to zbuf (the patch's
// C = q Cs entries hold the q slot rows, nr + 2 nc = q); the last CTA of the
// patch to finish (a ticket counter, reset by that CTA) mixes the slots back
// to the time nodes with V and writes y.  Every value is formed by one fixed
// sequence of operations, so the result does not depend on which CTA
// finishes last.
template <typename T, int Q, typename JOBS>
__global__ void __launch_bounds__(512) k_patch_apply_wide(const __grid_constant__ JOBS J) {
  using Vv = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  constexpr int CR = VEC / 2;
  constexpr int PF = 8; // loads of the inverse a thread keeps in flight
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nr = J.dc[0].nr, nc = J.dc[0].nc, ns = nr + nc;
  // CTA -> (job, patch of the job, slot)
  const long gp = blockIdx.x / ns;
  int jb = 0;
  if (sizeof(J.first) > 2 * sizeof(long)) // several jobs (a one-job table keeps jb = 0)
    while (gp >= J.first[jb + 1]) ++jb;
  const long p = gp - J.first[jb];
  const int a = (int)(blockIdx.x % ns); // slot of this CTA
  const DiagCoef<T> &dc = J.dc[jb];
  const int *__restrict__ pdofs = J.pdofs[jb];
  const T *__restrict__ res = J.res[jb];
  T *__restrict__ y = J.y[jb];
  T *__restrict__ zbuf = J.zbuf[jb];
  int *__restrict__ ticket = J.ticket[jb];
  const int Cs = J.pcs[jb][p];
  const long long doff = J.pdoff[jb][p];
  const bool cplx = a >= nr;
  const int nrg = cplx ? (Cs + CR - 1) / CR : (Cs + VEC - 1) / VEC; // row groups
  const int G = max(1, (int)blockDim.x / nrg);
  T *rs = reinterpret_cast<T *>(smem_raw); // [Q][Cs] gathered residual
  T *xr = rs + (size_t)Q * Cs;             // [Cs] slot input, real part
  T *xi = xr + Cs;                         // [Cs] imaginary part
  T *red = xi + Cs;                        // [G * nrg][VEC] partial sums
  const int t = threadIdx.x;
  const bool active = t < G * nrg;
  const int g = t % nrg, jg = t / nrg;
  const int ldR = (Cs + 3) / 4 * 4, ldC = 2 * ((Cs + 1) / 2 * 2);
  const T *Ab = J.pinv[jb] + J.pioff[jb][p];
  const Vv *col0 = cplx ? reinterpret_cast<const Vv *>(Ab + (size_t)nr * Cs * ldR + (size_t)(a - nr) * Cs * ldC +
                                                       2 * CR * g)
                        : reinterpret_cast<const Vv *>(Ab + (size_t)a * Cs * ldR + VEC * g);
  const long stride = (cplx ? ldC : ldR) / VEC;
  // the first PF columns of this thread are requested before the residual is
  // gathered, so that the two chains of loads overlap
  Vv buf[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u)
    if (active && jg + u * G < Cs) buf[u] = __ldcs(col0 + (long)(jg + u * G) * stride);
  for (int j = t; j < Q * Cs; j += blockDim.x) rs[j] = res[pdofs[doff + j]];
  __syncthreads();
  for (int m = t; m < Cs; m += blockDim.x) {
    T re = T(0), im = T(0);
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const T r = rs[b * Cs + m];
      re += dc.U[(a * Q + b) * 2] * r;
      im += dc.U[(a * Q + b) * 2 + 1] * r;
    }
    xr[m] = re;
    xi[m] = im;
  }
  __syncthreads();
  T vals[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) vals[v] = T(0);
  if (active) {
    for (int j0 = jg; j0 < Cs; j0 += PF * G) {
      Vv cur[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u) cur[u] = buf[u];
      // next PF columns in flight while these are used
#pragma unroll
      for (int u = 0; u < PF; ++u)
        if (j0 + (PF + u) * G < Cs) buf[u] = __ldcs(col0 + (long)(j0 + (PF + u) * G) * stride);
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int j = j0 + u * G;
        if (j >= Cs) break;
        if (!cplx) {
          fma_vec<T>(vals, cur[u], xr[j]);
        } else {
          const T *av = reinterpret_cast<const T *>(&cur[u]);
          const T ar = xr[j], ai = xi[j];
#pragma unroll
          for (int i = 0; i < CR; ++i) {
            vals[2 * i] += av[2 * i] * ar - av[2 * i + 1] * ai;
            vals[2 * i + 1] += av[2 * i] * ai + av[2 * i + 1] * ar;
          }
        }
      }
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) red[(size_t)t * VEC + v] = vals[v];
  }
  __syncthreads();
  // z rows of this slot: real slot a -> row a; complex slot -> rows
  // nr + 2 (a - nr) (re) and the next (im)
  T *z = zbuf + doff;
  for (int rg = t; rg < nrg; rg += blockDim.x) {
    T acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = red[(size_t)rg * VEC + v];
    for (int k = 1; k < G; ++k)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[v] += red[((size_t)k * nrg + rg) * VEC + v];
    if (!cplx) {
#pragma unroll
      for (int v = 0; v < VEC; ++v)
        if (VEC * rg + v < Cs) z[(size_t)a * Cs + VEC * rg + v] = acc[v];
    } else {
      const int row = nr + 2 * (a - nr);
#pragma unroll
      for (int i = 0; i < CR; ++i)
        if (CR * rg + i < Cs) {
          z[(size_t)row * Cs + CR * rg + i] = acc[2 * i];
          z[(size_t)(row + 1) * Cs + CR * rg + i] = acc[2 * i + 1];
        }
    }
  }
  if (ns > 1) {
    // the last CTA of the patch combines the slots (the flag is broadcast by
    // the barrier itself: no static shared memory beside the dynamic region)
    __threadfence();
    __syncthreads();
    int is_last = 0;
    if (t == 0) {
      is_last = atomicAdd(&ticket[p], 1) == ns - 1;
      if (is_last) ticket[p] = 0;
    }
    if (!__syncthreads_or(is_last)) return;
    __threadfence();
  } else {
    __syncthreads();
  }
  const int C = Q * Cs;
  for (int idx = t; idx < C; idx += blockDim.x) {
    const int b = idx / Cs, m = idx - b * Cs;
    T val = T(0);
    for (int s2 = 0; s2 < nr; ++s2) val += dc.V[(b * ns + s2) * 2] * __ldcg(z + (size_t)s2 * Cs + m);
    for (int c = 0; c < nc; ++c) {
      const int s2 = nr + c;
      val += T(2) * (dc.V[(b * ns + s2) * 2] * __ldcg(z + (size_t)(nr + 2 * c) * Cs + m) -
                     dc.V[(b * ns + s2) * 2 + 1] * __ldcg(z + (size_t)(nr + 2 * c + 1) * Cs + m));
    }
    y[doff + idx] = val;
  }
}

// d = (zero ? 0 : d) + scale * sum of the patch results holding each dof.
// scale = omega / (number of patches holding the dof): Algorithm 4.1's
// d = z / p written as d + omega D^{-1} sum_P E_P A_P^{-1} R_P (b - A d).
template <typename T>
__global__ void k_vanka_update(long N, const int *__restrict__ iptr, const int *__restrict__ ipos,
                               const T *__restrict__ scale, const T *__restrict__ y, T *__restrict__ d, int zero,
                               int nb, long ystride) {
  const int col = (int)(blockIdx.x % (unsigned)nb);
  const long i = (long)(blockIdx.x / (unsigned)nb) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  y += (long)col * ystride;
  d += (long)col * N;
  T acc = T(0);
  for (int e = iptr[i]; e < iptr[i + 1]; ++e) acc += y[ipos[e]];
  d[i] = (zero ? T(0) : d[i]) + scale[i] * acc;
}
