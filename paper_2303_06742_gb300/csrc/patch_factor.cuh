// Patch inverses of the time-diagonal form computed on the device (setup,
// Def. 4.2 / Eq. 4.13): for every patch P and eigenvalue slot a of W^{-1} Dt,
// (lam_a S1_P + S2_P)^{-1} in FP64 by Gauss-Jordan elimination with partial
// pivoting (first largest modulus in the column), written in the storage
// layout of the streaming kernel (column-major, ld = 4 ceil(Cs/4) for a real
// slot; (re, im) interleaved per row, ld = 2 * 2 ceil(Cs/2) for a complex
// slot), rounded to the storage type.  Included by stfem.cu.
//
// Persistent CTAs take (patch, slot) items from an atomic counter (patch
// sizes vary, so a static split would leave CTAs idle); the working matrix
// lives in a global scratch block of the CTA (L2-resident: the matrices of
// all CTAs in flight fit in L2), planar real / imaginary parts.
// No waits: every step ends at __syncthreads.  A zero or non-finite pivot
// marks the patch in *bad (the smallest such index wins) and the item stops.

constexpr int PF_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PF_THREADS)
    k_patch_factor(long p0, long np, int nr, int nc, const double *__restrict__ lam, const int *__restrict__ pcs,
                   const long long *__restrict__ boff, const double *__restrict__ blocks,
                   const long long *__restrict__ pioff, T *__restrict__ pinv, double *__restrict__ scratch,
                   long scr_stride, long long *__restrict__ bad, unsigned long long *__restrict__ next) {
  __shared__ double fr[512], fi[512]; // column k before the elimination (Cs <= 512)
  __shared__ double red_v[PF_THREADS];
  __shared__ int red_i[PF_THREADS];
  __shared__ int piv[512];
  __shared__ int stop;
  __shared__ long long take;
  const int ns = nr + nc;
  double *Zr = scratch + (long)blockIdx.x * scr_stride;
  for (;;) {
    if (threadIdx.x == 0) take = (long long)atomicAdd(next, 1ull);
    __syncthreads();
    const long item = (long)take;
    __syncthreads();
    if (item >= np * ns) break;
    const long pl = item / ns;  // patch within the batch
    const int a = (int)(item - pl * ns);
    const long p = p0 + pl;
    const int n = pcs[p];
    const bool cplx = a >= nr;
    double *Zi = Zr + (long)n * n;
    const double *S1 = blocks + boff[pl], *S2 = S1 + (long)n * n;
    const double lr = lam[2 * a], li = lam[2 * a + 1];
    for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) {
      Zr[e] = lr * S1[e] + S2[e];
      if (cplx) Zi[e] = li * S1[e];
    }
    if (threadIdx.x == 0) stop = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      // pivot: first row i >= k of largest modulus in column k
      double best = -1.0;
      int bi = n;
      for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        const double v = cplx ? hypot(Zr[(long)i * n + k], Zi[(long)i * n + k]) : fabs(Zr[(long)i * n + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      red_v[threadIdx.x] = best;
      red_i[threadIdx.x] = bi;
      __syncthreads();
      for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
          const double v2 = red_v[threadIdx.x + o];
          const int i2 = red_i[threadIdx.x + o];
          if (v2 > red_v[threadIdx.x] || (v2 == red_v[threadIdx.x] && i2 < red_i[threadIdx.x])) {
            red_v[threadIdx.x] = v2;
            red_i[threadIdx.x] = i2;
          }
        }
        __syncthreads();
      }
      const int pr = red_i[0];
      const double pv = red_v[0];
      if (!(pv > 0.0) || !isfinite(pv) || pr >= n) {
        if (threadIdx.x == 0) {
          stop = 1;
          atomicMin((unsigned long long *)bad, (unsigned long long)p);
        }
        __syncthreads();
        break;
      }
      if (threadIdx.x == 0) piv[k] = pr;
      if (pr != k)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          double t = Zr[(long)k * n + j];
          Zr[(long)k * n + j] = Zr[(long)pr * n + j];
          Zr[(long)pr * n + j] = t;
          if (cplx) {
            t = Zi[(long)k * n + j];
            Zi[(long)k * n + j] = Zi[(long)pr * n + j];
            Zi[(long)pr * n + j] = t;
          }
        }
      __syncthreads();
      // row k divided by the pivot, with the pivot entry replaced by 1
      const double dr = Zr[(long)k * n + k], di = cplx ? Zi[(long)k * n + k] : 0.0;
      const double den = dr * dr + di * di, ir = dr / den, ii = -di / den;
      __syncthreads();
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double x = j == k ? 1.0 : Zr[(long)k * n + j];
        const double y = j == k ? 0.0 : (cplx ? Zi[(long)k * n + j] : 0.0);
        Zr[(long)k * n + j] = x * ir - y * ii;
        if (cplx) Zi[(long)k * n + j] = x * ii + y * ir;
      }
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        fr[i] = Zr[(long)i * n + k];
        fi[i] = cplx ? Zi[(long)i * n + k] : 0.0;
      }
      __syncthreads();
      // every other row: z_i -= f_i z_k, with column k starting from 0
      for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e - (long)i * n);
        if (i == k) continue;
        const double f1 = fr[i], f2 = fi[i];
        if (f1 == 0.0 && f2 == 0.0) continue;
        const double x = Zr[(long)k * n + j], y = cplx ? Zi[(long)k * n + j] : 0.0;
        const double zr = j == k ? 0.0 : Zr[e];
        Zr[e] = zr - (f1 * x - f2 * y);
        if (cplx) {
          const double zi = j == k ? 0.0 : Zi[e];
          Zi[e] = zi - (f1 * y + f2 * x);
        }
      }
      __syncthreads();
    }
    if (stop) {
      __syncthreads();
      continue;
    }
    // undo the row interchanges on the columns, last first
    for (int k = n - 1; k >= 0; --k) {
      const int pk = piv[k];
      if (pk != k)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          double t = Zr[(long)i * n + k];
          Zr[(long)i * n + k] = Zr[(long)i * n + pk];
          Zr[(long)i * n + pk] = t;
          if (cplx) {
            t = Zi[(long)i * n + k];
            Zi[(long)i * n + k] = Zi[(long)i * n + pk];
            Zi[(long)i * n + pk] = t;
          }
        }
      __syncthreads();
    }
    // store: column j of the inverse at ld stride
    const int ldR = (n + 3) / 4 * 4, ldC = 2 * ((n + 1) / 2 * 2);
    T *dst = pinv + pioff[p] + (cplx ? (long)nr * n * ldR + (long)(a - nr) * n * ldC : (long)a * n * ldR);
    for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) {
      const int j = (int)(e / n), i = (int)(e - (long)j * n); // consecutive threads: consecutive rows i
      if (cplx) {
        dst[(long)j * ldC + 2 * i] = (T)Zr[(long)i * n + j];
        dst[(long)j * ldC + 2 * i + 1] = (T)Zi[(long)i * n + j];
      } else {
        dst[(long)j * ldR + i] = (T)Zr[(long)i * n + j];
      }
    }
    __syncthreads();
  }
}

// Tensor-core tiles (layout of tc_patch.cuh) from the FP32 time-diagonal
// inverses already on the device: one CTA per patch.
__global__ void k_build_tc_tiles(const int *__restrict__ pcs, const long long *__restrict__ pioff,
                                 const float *__restrict__ pinv, const long long *__restrict__ ptoff,
                                 float *__restrict__ ptile, int nr, int nc) {
  const long p = blockIdx.x;
  const int Cs = pcs[p], c8 = (Cs + 7) / 8 * 8;
  const int ldR = (Cs + 3) / 4 * 4, ldC = 2 * ((Cs + 1) / 2 * 2);
  const float *inv = pinv + pioff[p];
  float *t = ptile + ptoff[p];
  for (int a = 0; a < nr + nc; ++a) {
    const bool cplx = a >= nr;
    const int K = cplx ? 2 * c8 : c8;
    const float *z = cplx ? inv + (long)nr * Cs * ldR + (long)(a - nr) * Cs * ldC : inv + (long)a * Cs * ldR;
    for (long e = threadIdx.x; e < (long)K * c8; e += blockDim.x) {
      const int k = (int)(e / c8), m = (int)(e - (long)k * c8);
      float v = 0.f;
      if (m < Cs) {
        if (!cplx) {
          if (k < Cs) v = z[(long)k * ldR + m];
        } else {
          const int kk = k < c8 ? k : k - c8;
          if (kk < Cs) v = z[(long)kk * ldC + 2 * m + (k < c8 ? 0 : 1)];
        }
      }
      t[(long)(k / 8) * c8 * 8 + ((m / 8) * 2 + (k % 8) / 4) * 32 + (m % 8) * 4 + (k % 4)] = v;
    }
    t += (long)K * c8;
  }
}
