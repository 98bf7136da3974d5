// Transfers, the coarse solve and the FP64 BLAS-1 steps of FGMRES.  Included
// by stfem.cu inside its anonymous namespace, after the device helpers.

// ---------------------------------------------------------------- transfers
// out[a, blk, node*d + c] (+)= sum_e M[node, e] in[a, blk, col_e*d + c] for the
// vector blocks blk = V, U (scalar operator of the Q_r space) and
// out[a, P, node] (+)= sum_e Mp[node, e] in[a, P, col_e] (Q_{r-1} space).
// One thread per (time node, block, output node): the d components of a node
// are contiguous, so each operator entry feeds D loads from one segment.
template <typename T, int D, int G>
__global__ void k_transfer(long nu_out, long np_out, int q, long ns_out, long R_out, long ns_in, long R_in,
                           const int *__restrict__ up, const int *__restrict__ uc, const T *__restrict__ uv,
                           const int *__restrict__ pp, const int *__restrict__ pc, const T *__restrict__ pv,
                           const T *__restrict__ in, T *__restrict__ out, int add, int nb, long in_stride,
                           long out_stride) {
  // G lanes per output (the long rows of P^T in the restriction), reduced by
  // xor-shuffles in a fixed order; every lane of the warp takes part in the
  // shuffles (lanes without an output carry zeros)
  const int col = (int)(blockIdx.x % (unsigned)nb);
  const long gid = (long)(blockIdx.x / (unsigned)nb) * blockDim.x + threadIdx.x;
  const long i = gid / G;
  const int lane = (int)(gid % G);
  in += (long)col * in_stride;
  out += (long)col * out_stride;
  const long nuq = 2 * nu_out * q;
  T acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = T(0);
  int kind = 0;
  long node = 0;
  int a = 0, blk = 0;
  if (i < nuq) {
    kind = 1;
    node = i % nu_out;
    const long ab = i / nu_out; // a * 2 + blk
    a = (int)(ab >> 1);
    blk = (int)(ab & 1);
    const T *src = in + (long)a * ns_in + blk * R_in;
    for (int e = up[node] + lane; e < up[node + 1]; e += G) {
      const T w = uv[e];
      const T *sp = src + (long)uc[e] * D;
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] += w * sp[c];
    }
  } else if (i < nuq + np_out * q) {
    kind = 2;
    const long j = i - nuq;
    node = j % np_out;
    a = (int)(j / np_out);
    const T *src = in + (long)a * ns_in + 2 * R_in;
    for (int e = pp[node] + lane; e < pp[node + 1]; e += G) acc[0] += pv[e] * src[pc[e]];
  }
  if (G > 1) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, G);
  }
  if (lane != 0) return;
  if (kind == 1) {
    T *dst = out + (long)a * ns_out + blk * R_out + node * D;
#pragma unroll
    for (int c = 0; c < D; ++c) dst[c] = add ? dst[c] + acc[c] : acc[c];
  } else if (kind == 2) {
    T *dst = out + (long)a * ns_out + 2 * R_out + node;
    *dst = add ? *dst + acc[0] : acc[0];
  }
}

// ---------------------------------------------------------------- coarse
// x = Ainv b with a dense FP64 inverse (one warp per row).
template <typename T>
__global__ void k_coarse(long n, const double *__restrict__ Ainv, const T *__restrict__ b, T *__restrict__ x,
                         int nb) {
  const int col = (int)(blockIdx.x % (unsigned)nb);
  const long row = ((long)(blockIdx.x / (unsigned)nb) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  b += (long)col * n;
  x += (long)col * n;
  double acc = 0.0;
  const double *a = Ainv + row * n;
  for (long j = lane; j < n; j += 32) acc += a[j] * (double)b[j];
  acc = warp_sum(acc);
  if (lane == 0) x[row] = (T)acc;
}

template <typename A, typename B>
__global__ void k_convert(long n, const A *__restrict__ a, B *__restrict__ b) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

// b[c * sb + i] = a[c * sa + i] for nb columns of n entries (with conversion)
template <typename A, typename B>
__global__ void k_copy_cols(long n, int nb, const A *__restrict__ a, long sa, B *__restrict__ b, long sb) {
  const int col = (int)(blockIdx.x % (unsigned)nb);
  const long i = (long)(blockIdx.x / (unsigned)nb) * blockDim.x + threadIdx.x;
  if (i < n) b[(long)col * sb + i] = (B)a[(long)col * sa + i];
}

// ---------------------------------------------------------------- BLAS-1 (FP64)
// (the dot products run 4 blocks per SM: stfem_ctx::dot_blocks)
constexpr int DOT_THREADS = 256;
constexpr int DOT_NV = 8;

// partial[v][block] = sum over the block's share of V_v . w  (v < k)
__global__ void __launch_bounds__(DOT_THREADS) k_multidot(int k, const double *__restrict__ V, long ldV,
                                                          const double *__restrict__ w, long n,
                                                          double *__restrict__ partial) {
  const int v0 = blockIdx.y * DOT_NV;
  double acc[DOT_NV];
#pragma unroll
  for (int t = 0; t < DOT_NV; ++t) acc[t] = 0.0;
  // two entries per trip: twice the independent loads in flight
  const long stride = (long)gridDim.x * blockDim.x;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
    const long i2 = i + stride;
    const bool two = i2 < n;
    const double wi = w[i], wi2 = two ? w[i2] : 0.0;
#pragma unroll
    for (int t = 0; t < DOT_NV; ++t)
      if (v0 + t < k) {
        const double a = V[(long)(v0 + t) * ldV + i], a2 = two ? V[(long)(v0 + t) * ldV + i2] : 0.0;
        acc[t] += a * wi + a2 * wi2;
      }
  }
  __shared__ double sm[DOT_NV][DOT_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < DOT_NV; ++t) {
    const double s = warp_sum(acc[t]);
    if (lane == 0) sm[t][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < DOT_NV; ++t) {
      double s = lane < DOT_THREADS / 32 ? sm[t][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0 && v0 + t < k) partial[(long)(v0 + t) * gridDim.x + blockIdx.x] = s;
    }
  }
}

// w <- w - sum_v h[v] V_v, fused with the block partial sums of the next
// Gram-Schmidt quantity: mode 0, partial[v][block] = V_v . w_new (v < k);
// mode 1, partial[0][block] = w_new . w_new.  KB >= k bounds the register
// accumulators.
template <int KB>
__global__ void __launch_bounds__(DOT_THREADS) k_axpy_dot(int k, const double *__restrict__ V, long ldV,
                                                          const double *__restrict__ h, double *__restrict__ w,
                                                          long n, double *__restrict__ partial, int mode) {
  double acc[KB];
#pragma unroll
  for (int t = 0; t < KB; ++t) acc[t] = 0.0;
  double hv[KB];
#pragma unroll
  for (int t = 0; t < KB; ++t) hv[t] = t < k ? h[t] : 0.0;
  // small blocks take two entries per trip (more independent loads in flight)
  constexpr int UN = KB <= 8 ? 2 : 1;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += UN * stride) {
    double vi[UN][KB], wn[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const long i = i0 + u * stride;
      const bool in = i < n;
      double s = 0.0;
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        vi[u][t] = (t < k && in) ? V[(long)t * ldV + i] : 0.0;
        s += hv[t] * vi[u][t];
      }
      wn[u] = in ? w[i] - s : 0.0;
    }
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const long i = i0 + u * stride;
      if (i < n) w[i] = wn[u];
      if (mode == 0) {
#pragma unroll
        for (int t = 0; t < KB; ++t) acc[t] += vi[u][t] * wn[u];
      } else {
        acc[0] += wn[u] * wn[u];
      }
    }
  }
  __shared__ double sm[KB][DOT_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nout = mode == 0 ? k : 1;
#pragma unroll
  for (int t = 0; t < KB; ++t) {
    const double sv = warp_sum(acc[t]);
    if (lane == 0) sm[t][warp] = sv;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      double sv = lane < DOT_THREADS / 32 ? sm[t][lane] : 0.0;
      sv = warp_sum(sv);
      if (lane == 0 && t < nout) partial[(long)t * gridDim.x + blockIdx.x] = sv;
    }
  }
}

// out[v] = sum_b partial[v][b] in a fixed order (one block per v).
__global__ void k_reduce_partials(int nb, const double *__restrict__ partial, double *__restrict__ out) {
  __shared__ double sm[32];
  const int v = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(long)v * nb + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[v] = t;
  }
}

// w -= sum_v h[v] V_v
__global__ void k_multiaxpy(int k, const double *__restrict__ V, long ldV, const double *__restrict__ h,
                            double *__restrict__ w, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int v = 0; v < k; ++v) acc += h[v] * V[(long)v * ldV + i];
  w[i] -= acc;
}

// dst = src / *div  (or src / div_host when div == nullptr)
__global__ void k_div(long n, const double *__restrict__ src, double *__restrict__ dst, const double *div,
                      double div_host) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = div ? *div : div_host;
  dst[i] = s != 0.0 ? src[i] / s : 0.0; // a zero column (finished right-hand side) stays zero
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes, the
// previous Givens rotations applied, a new rotation for (H_jj, H_{j+1,j})
// and the update of g.  status = {|g_{j+1}|, h_{j+1,j}}.
__global__ void k_givens(int j, int m1, const double *__restrict__ h1, const double *__restrict__ h2,
                         const double *__restrict__ hn2, double *__restrict__ H, double *__restrict__ cs,
                         double *__restrict__ sn, double *__restrict__ g, double *__restrict__ hnorm,
                         double *__restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double col[MAXM + 1];
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  const double hn = sqrt(*hn2);
  col[j + 1] = hn;
  *hnorm = hn;
  for (int i = 0; i < j; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = col[j], b = col[j + 1];
  const double rho = hypot(a, b);
  cs[j] = rho != 0.0 ? a / rho : 1.0;
  sn[j] = rho != 0.0 ? b / rho : 0.0;
  col[j] = rho;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  for (int i = 0; i <= j + 1; ++i) H[(long)j * m1 + i] = col[i];
  status[0] = fabs(g[j + 1]);
  status[1] = hn;
}

// Back substitution H(0:k,0:k) y = g(0:k).
__global__ void k_backsolve(int k, int m1, const double *__restrict__ H, const double *__restrict__ g,
                            double *__restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = 0.0;
    for (int l = i + 1; l < k; ++l) s += H[(long)l * m1 + i] * y[l];
    y[i] = (g[i] - s) / H[(long)i * m1 + i];
  }
}

template <typename TZ>
__global__ void k_update_x(long n, int k, const TZ *__restrict__ Z, long ldZ, const double *__restrict__ y,
                           double *__restrict__ x) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int j = 0; j < k; ++j) acc += (double)Z[(long)j * ldZ + i] * y[j];
  x[i] += acc;
}

__global__ void k_set(double *p, double v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

__global__ void k_repeat(long ns, int q, const double *__restrict__ state, double *__restrict__ x) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns * q) return;
  x[i] = state[i % ns];
}
