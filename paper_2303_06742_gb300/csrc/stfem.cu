// GB300 (sm_103a) implementation of the GMRES-GMG solver for the space-time
// FEM of dynamic poro-/thermoelasticity (arXiv 2303.06742) behind the C ABI
// declared in include/stfem.h.
//
// Data layout in HBM: slab vectors in the paper's order (Eq. 4.4), time node
// outermost, so that each spatial row of the Kronecker SpMV reads the q time
// values of a column with q coalesced gathers.  Each level holds one spatial
// CSR with two values per entry (coefficients of Dt and of W), the patch dof
// lists and the patch inverses stored column-major (a thread owns VEC
// consecutive rows and streams the inverse with 16-byte loads), and an inverse
// map dof -> (patch, local row) for the deterministic averaged update.
#include "../../include/stfem.h"
#include "fem.hpp"
#include "kernels.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <climits>
#include <array>
#include <chrono>
#include <future>
#include <map>
#include <memory>
#include <tuple>
#include <vector>

using namespace stfem_dev;

// Launch-shape tuning of the patch apply (compile-time constants).
#ifndef STFEM_DIAG_UNROLL_COMPLEX
#define STFEM_DIAG_UNROLL_COMPLEX 0
#endif
#ifndef STFEM_STREAM_MIN_PATCHES
// time-diagonal levels with fewer patches use the one-CTA-per-patch kernel
// with column groups (more loads in flight per patch) instead of streaming
#define STFEM_STREAM_MIN_PATCHES 0
#endif
// lanes per output of the restriction (rows of P^T hold up to (2r+1)^d
// entries) and of the prolongation (rows of P: up to (r+1)^d); measured on
// both bench workloads: 8 lanes for the restriction took 5% off a 2D slab
#ifndef STFEM_RESTRICT_LANES
#define STFEM_RESTRICT_LANES 8
#endif
#ifndef STFEM_PROLONG_LANES
#define STFEM_PROLONG_LANES 1
#endif
#ifndef STFEM_PATCH_THREADS_PER_SM
#define STFEM_PATCH_THREADS_PER_SM 4096
#endif

namespace {

// ============================================================ device helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

#include "spmv.cuh"
#include "matfree.cuh"
#include "vanka.cuh"

// ---------------------------------------------------------------- bulk-copy streaming
// Helpers for the asynchronous bulk copy (cp.async.bulk) of contiguous global
// data into shared memory, completed on an mbarrier (transaction bytes).
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(smem_addr(bar)), "r"(parity)
               : "memory");
  return ok != 0;
}
// Waits until the phase of the given parity has completed, for at most
// `limit` clock cycles; false on timeout (the caller then aborts).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

constexpr int STREAM_STAGES = 12;                   // most stages of the ring (runtime: nst)
constexpr int STREAM_CHUNK = 16384;                 // bytes per shared-memory stage
// Ring shapes {stages, CTAs per SM, patch tile} the autotuners time: shallow
// rings with many CTAs per SM for levels with many patches, deep rings (up to
// the whole of a patch's inverses in flight) with one or two CTAs per SM for
// levels with a few patches per SM, where a CTA's own latency bounds the level.
#define STREAM_SHAPE_CANDIDATES                                                                                    \
  {{2, 5, 1}, {3, 4, 1}, {4, 3, 1}, {2, 5, 2}, {4, 3, 2}, {4, 3, 4}, {6, 3, 1}, {8, 2, 1}, {12, 1, 1}}
// clock cycles a drain of copies in flight may wait (about 2 s at 2 GHz);
// the other waits take the handle's limit (stfem_set_wait_limit)
constexpr long long STREAM_WAIT_LIMIT = 4000000000LL;
// shared-memory bytes before the per-patch vectors: the ring, the barriers
__host__ __device__ constexpr int stream_header(int nst) { return nst * STREAM_CHUNK + 2 * STREAM_STAGES * 8 + 16; }

// Patch sets processed by one launch of a patch-apply kernel: `njobs` levels
// (of one handle, or of several handles that advance together), job j holding
// the global patches [first[j], first[j + 1]).  Passed by value
// (__grid_constant__): the launch carries it, so a captured graph replays it.
// All jobs have the same number of time nodes (hence the same slot structure
// nr, nc); their U, V factors may differ (they depend on tau).
template <typename T, int MAXJ>
struct PatchJobs {
  int njobs;
  long first[MAXJ + 1];
  const int *pcs[MAXJ];
  const long long *pdoff[MAXJ];
  const int *pdofs[MAXJ];
  const long long *pioff[MAXJ];
  const T *pinv[MAXJ];
  const T *res[MAXJ];
  T *y[MAXJ];
  T *zbuf[MAXJ];  // wide kernel: slot results
  int *ticket[MAXJ];
  DiagCoef<T> dc[MAXJ];
};
constexpr int MAXJOBS = 16; // levels one fused launch takes

// Time-diagonal patch apply (see k_patch_apply_diag) with the inverse blocks
// streamed by bulk copies.  Persistent CTAs take tiles of `tile` consecutive
// patches: patches b * tile .. b * tile + tile - 1, then the same plus
// gridDim.x * tile, ... over the patches of all jobs (so one launch may serve
// the levels of several handles).  The last warp is the producer: one lane
// walks the (patch, slot, column chunk) sequence and copies each chunk
// (contiguous, 16-byte aligned, a multiple of 16 bytes) into a ring of
// nst <= STREAM_STAGES shared stages.  The other warps gather and mix the
// residual, consume the chunks of their slot rows from shared memory, and mix
// the result back.  A patch's arithmetic does not depend on the CTA, the tile
// or the other jobs of the launch.
// Every wait is bounded by `wait` clock cycles; on a timeout the CTA sets
// *err, the producer waits (bounded by STREAM_WAIT_LIMIT) for its copies still
// in flight, and the CTA returns.  stall != 0 makes the producer issue no copy
// at all, so that every consumer's first wait runs out (the failure-detection
// test of the bounded waits: nothing is in flight when the CTA leaves).
template <typename T, int Q, int MAXJ>
__global__ void __launch_bounds__(1024) k_patch_apply_stream(const __grid_constant__ PatchJobs<T, MAXJ> J, int maxCs,
                                                             int tile, int *__restrict__ err, int nst,
                                                             long long wait, int stall) {
  using Vv = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  constexpr int CR = VEC / 2;
  extern __shared__ __align__(128) unsigned char smem_stream[];
  unsigned char *stage = smem_stream;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_stream + nst * STREAM_CHUNK);
  uint64_t *empty = full + STREAM_STAGES;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + STREAM_STAGES);
  const int nr = J.dc[0].nr, nc = J.dc[0].nc, ns = nr + nc, nrow = nr + 2 * nc;
  const long npatch = J.first[J.njobs];
  T *rs = reinterpret_cast<T *>(smem_stream + stream_header(nst));
  T *rt = rs + (size_t)Q * maxCs;
  T *z = rt + (size_t)nrow * maxCs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwc = (blockDim.x >> 5) - 1; // consumer warps
  const int nct = nwc * 32;
  if (threadIdx.x == 0) {
    for (int st = 0; st < nst; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], nwc);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long step = (long)gridDim.x * tile;

  if (warp == nwc) {
    // ---------------- producer
    if (lane != 0 || stall) return;
    long long it = 0;
    bool ok = true;
    int j = 0;
    for (long b = (long)blockIdx.x * tile; b < npatch && ok; b += step)
      for (long p = b; p < b + tile && p < npatch && ok; ++p) {
        if (MAXJ > 1)
          while (p >= J.first[j + 1]) ++j;
        const long lp = p - J.first[j];
        const int Cs = J.pcs[j][lp];
        const int ldR = (Cs + 3) / 4 * 4, ldC = 2 * ((Cs + 1) / 2 * 2);
        const T *base = J.pinv[j] + J.pioff[j][lp];
        for (int sl = 0; sl < ns && ok; ++sl) {
          const int ld = sl < nr ? ldR : ldC;
          const T *sb =
              base + (sl < nr ? (size_t)sl * Cs * ldR : (size_t)nr * Cs * ldR + (size_t)(sl - nr) * Cs * ldC);
          const int K = max(1, STREAM_CHUNK / (ld * (int)sizeof(T)));
          for (int j0 = 0; j0 < Cs; j0 += K) {
            const int st = (int)(it % nst);
            if (it >= nst && !mbar_wait(&empty[st], (uint32_t)(((it / nst) - 1) & 1), wait)) {
              ok = false;
              break;
            }
            if (*abort_flag) {
              ok = false;
              break;
            }
            const uint32_t bytes = (uint32_t)(min(K, Cs - j0) * ld * (int)sizeof(T));
            mbar_arrive_expect_tx(&full[st], bytes);
            bulk_copy_g2s(stage + (size_t)st * STREAM_CHUNK, sb + (size_t)j0 * ld, bytes, &full[st]);
            ++it;
          }
        }
      }
    if (!ok) {
      atomicExch(err, 1);
      *abort_flag = 1;
      // copies still in flight must land before the CTA exits
      for (long long k = (it > nst ? it - nst : 0); k < it; ++k)
        mbar_wait(&full[k % nst], (uint32_t)((k / nst) & 1), STREAM_WAIT_LIMIT);
    }
    return;
  }

  // ---------------- consumers (threads 0 .. nct-1)
  const int tid = threadIdx.x;
  long long it = 0;
  int j = 0;
  // The first PFK gather entries of a thread for the CTA's next patch are
  // loaded into registers while the current patch streams, so the gather's two
  // dependent loads overlap the copies (the values are the same as a direct
  // gather's).
  constexpr int PFK = 4;
  T pre[PFK];
  bool have_pre = false;
  auto prefetch = [&](long pn) {
    int jn = j;
    if (MAXJ > 1)
      while (pn >= J.first[jn + 1]) ++jn;
    const long lpn = pn - J.first[jn];
    const int Cn = Q * J.pcs[jn][lpn];
    const long long dn = J.pdoff[jn][lpn];
    const int *__restrict__ pd = J.pdofs[jn];
    const T *__restrict__ rr = J.res[jn];
#pragma unroll
    for (int k = 0; k < PFK; ++k)
      if (tid + k * nct < Cn) pre[k] = rr[pd[dn + tid + k * nct]];
  };
  for (long b = (long)blockIdx.x * tile; b < npatch; b += step)
    for (long p = b; p < b + tile && p < npatch; ++p) {
      // all consumers pass the same barriers, so they all see the flag and
      // leave together (no barrier is left waiting)
      consumer_sync(nct);
      if (*abort_flag) return;
      if (MAXJ > 1) // one job: j stays 0 and the factors are launch constants
        while (p >= J.first[j + 1]) ++j;
      const long lp = p - J.first[j];
      const DiagCoef<T> &dc = J.dc[j];
      const int Cs = J.pcs[j][lp], C = Q * Cs;
      const long long doff = J.pdoff[j][lp];
      const int *__restrict__ pdofs = J.pdofs[j];
      const T *__restrict__ res = J.res[j];
      T *__restrict__ y = J.y[j];
      {
        int jj = tid;
        if (have_pre) {
#pragma unroll
          for (int k = 0; k < PFK; ++k, jj += nct)
            if (jj < C) rs[jj] = pre[k];
        }
        for (; jj < C; jj += nct) rs[jj] = res[pdofs[doff + jj]];
      }
      consumer_sync(nct);
      for (int m = tid; m < Cs; m += nct) {
        for (int a = 0; a < ns; ++a) {
          T re = T(0), im = T(0);
#pragma unroll
          for (int bq = 0; bq < Q; ++bq) {
            const T r = rs[bq * Cs + m];
            re += dc.U[(a * Q + bq) * 2] * r;
            im += dc.U[(a * Q + bq) * 2 + 1] * r;
          }
          if (a < nr) {
            rt[a * Cs + m] = re;
          } else {
            rt[(nr + 2 * (a - nr)) * Cs + m] = re;
            rt[(nr + 2 * (a - nr) + 1) * Cs + m] = im;
          }
        }
      }
      consumer_sync(nct);
      {
        long pn = p + 1;
        if (!(pn < b + tile && pn < npatch)) pn = b + step;
        have_pre = pn < npatch;
        if (have_pre) prefetch(pn);
      }
      const int nRr = (Cs + VEC - 1) / VEC, nCr = (Cs + CR - 1) / CR;
      const int ldR = (Cs + 3) / 4 * 4, ldC = 2 * ((Cs + 1) / 2 * 2);
      int role = -1, slot = 0, m0 = 0;
      if (tid < nr * nRr) {
        role = 0;
        slot = tid / nRr;
        m0 = VEC * (tid % nRr);
      } else if (tid < nr * nRr + nc * nCr) {
        role = 1;
        const int t2 = tid - nr * nRr;
        slot = t2 / nCr;
        m0 = CR * (t2 % nCr);
      }
      T vals[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) vals[v] = T(0);
      for (int sl = 0; sl < ns; ++sl) {
        const int ld = sl < nr ? ldR : ldC;
        const int K = max(1, STREAM_CHUNK / (ld * (int)sizeof(T)));
        for (int j0 = 0; j0 < Cs; j0 += K) {
          const int st = (int)(it % nst);
          bool ready = !*abort_flag;
          if (ready && !mbar_wait(&full[st], (uint32_t)((it / nst) & 1), wait)) {
            atomicExch(err, 2);
            *abort_flag = 1;
            ready = false;
          }
          const int ncol = ready ? min(K, Cs - j0) : 0;
          const T *sbuf = reinterpret_cast<const T *>(stage + (size_t)st * STREAM_CHUNK);
          if (sl < nr) {
            if (role == 0 && slot == sl) {
              const T *x = rt + sl * Cs + j0;
              for (int jc = 0; jc < ncol; ++jc)
                fma_vec<T>(vals, *reinterpret_cast<const Vv *>(sbuf + (size_t)jc * ld + m0), x[jc]);
            }
          } else if (role == 1 && slot == sl - nr) {
            const T *xr = rt + (nr + 2 * slot) * Cs + j0, *xi = xr + Cs;
            for (int jc = 0; jc < ncol; ++jc) {
              const Vv a = *reinterpret_cast<const Vv *>(sbuf + (size_t)jc * ld + 2 * m0);
              const T *av = reinterpret_cast<const T *>(&a);
              const T ar = xr[jc], ai = xi[jc];
#pragma unroll
              for (int i = 0; i < CR; ++i) {
                vals[2 * i] += av[2 * i] * ar - av[2 * i + 1] * ai;
                vals[2 * i + 1] += av[2 * i] * ai + av[2 * i + 1] * ar;
              }
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[st]);
          ++it;
        }
      }
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
      consumer_sync(nct);
      for (int idx = tid; idx < C; idx += nct) {
        const int bq = idx / Cs, m = idx - bq * Cs;
        T val = T(0);
        for (int a = 0; a < nr; ++a) val += dc.V[(bq * ns + a) * 2] * z[a * Cs + m];
        for (int c = 0; c < nc; ++c) {
          const int a = nr + c;
          val += T(2) * (dc.V[(bq * ns + a) * 2] * z[(nr + 2 * c) * Cs + m] -
                         dc.V[(bq * ns + a) * 2 + 1] * z[(nr + 2 * c + 1) * Cs + m]);
        }
        y[doff + idx] = val;
      }
      consumer_sync(nct);
    }
}

#include "tc_patch.cuh"
#include "patch_factor.cuh"

#include "solver_kernels.cuh"
#include "problem_data.cuh"

// ============================================================ host side
inline int grid_for(long n, int threads) { return (int)((n + threads - 1) / threads); }

template <typename T>
struct DLevel {
  long ns = 0, N = 0, R = 0, S = 0;
  long long nnz = 0;
  // node-block operator (see k_spmv_nb)
  NodeBlockDev<T> nb{};
  // the same values as float pairs (see k_spmv_df; finest FP64 level, MIXED)
  NodeBlockDev<float2> nbdf{};
  // Problem B.1: -Cvol in the layout of nb.pu_c (assembled levels)
  const T *pu_cvol = nullptr;
  // matrix-free form of the same operator (finest FP32 level; see
  // matfree.cuh) and whether the level's single-column products use it
  bool has_mf = false, use_mf = false;
  MfDev mf{};
  double mf_bytes = 0.0, mf_flops = 0.0;
  bool has_df = false;
  double nb_bytes = 0.0, nb_flops = 0.0;
  // patches
  long npatch = 0;
  int maxC = 0;
  int *psize = nullptr, *pld = nullptr, *pdofs = nullptr;
  long long *pdoff = nullptr, *pioff = nullptr;
  T *pinv = nullptr;
  long long inv_elems = 0, sumC = 0;
  int *iptr = nullptr, *ipos = nullptr;
  T *scale = nullptr, *ybuf = nullptr;
  double patch_bytes = 0.0, patch_flops = 0.0; // algorithmic, per patch-apply launch
  double patch_inv_bytes = 0.0;                 // the inverse part of patch_bytes
  // tensor-core layout of the time-diagonal inverses (FP32 levels of
  // handles set up for several right-hand sides)
  // tc_nst_deep: the ring of a level with at most one patch per SM, which
  // runs one CTA per SM and so has the SM's shared memory to itself
  int tc = 0, tc_nst = 0, tc_nst_deep = 0;
  // ring shape of the streaming patch apply picked by autotune_stream (0: by
  // dimension)
  int tune_nst = 0, tune_cap = 0, tune_tile = 0;
  // levels with few patches use k_patch_apply_wide: its slot results (sumC
  // per column) and per-patch ticket counters
  int wide = 0;
  T *zbuf = nullptr;
  int *ticket = nullptr;
  uint32_t tc_cols = 0;
  long long *ptoff = nullptr;
  float *ptile = nullptr;
  // work items of the tensor-core apply (see tc_patch.cuh): [0] whole
  // patches, [1] single 128-row M tiles, each list largest first; which list
  // and which ring (tc_deep: one CTA per SM with the deepest ring) a launch
  // uses is picked by autotune_tc
  int2 *tc_items[2] = {nullptr, nullptr};
  long tc_nitem[2] = {0, 0};
  int tc_split = 0, tc_deep = 0;
  int form = 0;       // 0 dense inverses, 1 time-diagonal form
  int *pcs = nullptr; // spatial patch size Cs (form 1)
  int maxCs = 0;
  DiagCoef<T> dc{};
  double transfer_bytes = 0.0, transfer_nnz = 0.0;
  // work vectors: ncols columns of N (b, d, r) and of sumC (ybuf)
  T *b = nullptr, *d = nullptr, *r = nullptr;
  int ncols = 1;
  // transfer from level l-1 (valid for l >= 1): P rows fine, R rows coarse
  int *Pu_p = nullptr, *Pu_c = nullptr, *Pp_p = nullptr, *Pp_c = nullptr;
  int *Ru_p = nullptr, *Ru_c = nullptr, *Rp_p = nullptr, *Rp_c = nullptr;
  T *Pu_v = nullptr, *Pp_v = nullptr, *Ru_v = nullptr, *Rp_v = nullptr;
};

} // namespace

struct stfem_ctx {
  std::string err;
  cudaStream_t stream = 0;
  int device = 0;
  // streaming multiprocessors of the device (grid sizes of the persistent
  // kernels and of the dot products) and its SM clock (kHz)
  int nsm = 152, clock_khz = 2070000, dot_blocks = 4 * 152;
  // most CTAs of the persistent patch-apply kernels (0: as many as fit)
  int launch_cap = 0;
  // clock cycles a bounded wait of the streaming patch apply may take before
  // it reports a timeout; stall_copies != 0 makes its producer issue no copy
  long long wait_cycles = 4000000000LL;
  int stall_copies = 0;
  // recorded on the handle's stream before a fused launch of a group
  cudaEvent_t grp_ev = nullptr;
  // patch-apply kernel of the time-diagonal levels (STFEM_PATCH_KERNEL_*)
  int patch_kernel = 0;
  // operator of the finest FP32 level (STFEM_OPERATOR_*)
  int fine_op = 0;
  int dim = 2, r = 2, k = 1, q = 2, nlev = 1;
  double tau = 0.01, t0 = 0.0;
  int problem = 0;
  stfem::Temporal T;
  std::vector<stfem::Level> hl;
  std::vector<stfem::CSR> Pu, Pp; // index l: from l-1 to l
  ProbDev prob{};
  GeomDev geom{}; // finest level
  // FP64 operators of every level (built by stfem_setup)
  std::vector<DLevel<double>> L64;
  // FP32 V-cycle levels (built by gmg_setup in STFEM_MIXED)
  std::vector<DLevel<float>> L32;
  int precision = -1;
  double omega = 0.7;
  int nsweeps = 1;
  int patch_kind = STFEM_PATCHES_VERTEX, update = STFEM_UPDATE_AVERAGE;
  int stop = STFEM_STOP_RELATIVE;
  double *coarse_inv = nullptr;
  // FGMRES workspace
  int mcap = 0;
  double *V = nullptr, *Zd = nullptr, *w = nullptr, *rvec = nullptr, *zt = nullptr;
  float *Zf = nullptr;
  double *h1 = nullptr, *h2 = nullptr, *hn2 = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr,
         *y = nullptr, *hnorm = nullptr, *partial = nullptr, *status = nullptr;
  double *status_host = nullptr;
  int *dev_err = nullptr; // set by kernels whose bounded waits timed out
  // march buffers and load tables
  double *rhs = nullptr, *xs = nullptr, *ys = nullptr, *chi = nullptr, *tnode = nullptr, *src = nullptr;
  LoadTables lt{};
  std::vector<double> hist;
  std::vector<void *> allocs;
  long long device_bytes = 0; // sum of the handle's allocations
  // launch accounting: totals per kernel class; event pairs when profiling
  long long launches = 0;
  bool prof = false;
  struct KStat {
    long long launches = 0;
    double bytes = 0.0, flops = 0.0, ms = 0.0;
  } kstat[STFEM_KCLASS_COUNT];
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  // one captured CUDA graph per FGMRES iteration index j (same buffers every
  // solve), with the launch accounting of its kernels
  struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    KStat delta[STFEM_KCLASS_COUNT];
  };
  std::vector<GraphRec> graphs;
  bool use_graphs = true;
  std::vector<std::pair<int, size_t>> pending; // (class, index of start event)
  // several right-hand sides solved together: one FGMRES per column, all
  // columns preconditioned by one batched V-cycle
  int nrhs_cap = 1;
  struct Batch {
    int nb = 0, m = 0;
    long sw = 0; // stride of the per-column small arrays
    double *V = nullptr, *Zd = nullptr, *zt = nullptr, *w = nullptr, *rvec = nullptr, *rhs = nullptr,
           *xs = nullptr;
    float *Zf = nullptr;
    double *small = nullptr;  // per column: H, cs, sn, g, y, h1, h2, hnorm
    double *norms = nullptr;  // [nb] squared norms, then [nb][2] statuses
    double *host = nullptr;   // pinned copy of norms
    std::vector<GraphRec> graphs;
  } bt;
};

namespace {

// message of the last failed stfem_setup of the calling thread (setups of
// concurrent requests run on different threads)
thread_local std::string g_setup_err;

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                                   \
      return e_ == cudaErrorMemoryAllocation ? STFEM_ERR_OOM : STFEM_ERR_CUDA;                       \
    }                                                                                                \
  } while (0)

#define CKR(expr)                                                                                    \
  do {                                                                                               \
    int rc_ = (expr);                                                                                \
    if (rc_ < 0) return rc_;                                                                         \
  } while (0)

// Counts a kernel launch of class kc with its algorithmic bytes/flops and,
// when profiling is on, brackets it with a pair of events on the stream.
struct Launch {
  stfem_h h;
  int kc;
  Launch(stfem_h h_, int kc_, double bytes, double flops) : h(h_), kc(kc_) {
    h->launches++;
    h->kstat[kc].launches++;
    h->kstat[kc].bytes += bytes;
    h->kstat[kc].flops += flops;
    if (h->prof) record();
  }
  ~Launch() {
    if (h->prof) record();
  }
  void record() {
    if (h->evnext >= h->evpool.size()) {
      for (int i = 0; i < 1024; ++i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->evpool.push_back(e);
      }
    }
    if (h->evnext % 2 == 0) h->pending.push_back({kc, h->evnext});
    cudaEventRecord(h->evpool[h->evnext++], h->stream);
  }
};

template <typename T>
int dalloc(stfem_h h, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  CK(cudaMalloc((void **)p, n * sizeof(T)));
  h->allocs.push_back((void *)*p);
  h->device_bytes += (long long)(n * sizeof(T));
  return 0;
}

// src: any contiguous container (std::vector, stfem::hvec); copied as is
// when the element types agree, else converted on the host (threaded)
template <typename T, typename V>
int upload(stfem_h h, T **p, const V &src) {
  using S = typename V::value_type;
  CKR(dalloc(h, p, src.size()));
  if (src.empty()) return 0;
  if (std::is_same<T, S>::value) {
    CK(cudaMemcpy(*p, (const void *)src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return 0;
  }
  stfem::hvec<T> tmp(src.size());
  const long n = (long)src.size();
  const S *in = src.data();
  T *o = tmp.data();
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) o[i] = (T)in[i];
  CK(cudaMemcpy(*p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  return 0;
}

template <typename T>
TimeCoef<T> time_coef(const stfem::Temporal &Tm, double tau) {
  TimeCoef<T> tc{};
  tc.q = Tm.q;
  for (int i = 0; i < Tm.q * Tm.q; ++i) tc.Dt[i] = (T)Tm.Dt[i];
  for (int b = 0; b < Tm.q; ++b) tc.W[b] = (T)(0.5 * tau * Tm.w[b]);
  return tc;
}

// Lanes per node: the FP64 instance is bound by the FP64 pipe, so fewer lanes
// (fewer FP64 shuffle-reduction adds); the FP32 instances are latency-bound,
// so more lanes for the long 3D rows (up to 125 neighbours).
template <typename T, int D>
struct SpmvLanes {
  static constexpr int G = sizeof(T) == 8 ? 2 : (D == 3 ? 8 : 4);
};

// A level whose nodes fill at most about two waves of the GPU with a warp
// per node (the coarse levels of the V-cycle) takes 32 lanes per node: each
// lane then walks one or two neighbours instead of a dependent chain of ten
// or more.  A fixed rule on the level's size, so a level's arithmetic never
// depends on the run.
template <typename T>
bool spmv_wide_lanes(const DLevel<T> &L, int nsm) {
  return (L.nb.nu + L.nb.np) * 32 <= (long)nsm * 1024;
}

template <typename T, int Q, int D, int G>
void launch_spmv_qdg(cudaStream_t s, const DLevel<T> &L, const TimeCoef<T> &tc, const T *x, const T *rhs, T *y,
                     int mode, int nb) {
  const long threads = (L.nb.nu + L.nb.np) * G;
  // several FP32 columns: two per thread (a node block loaded once serves
  // both; per column the same sums in the same order)
  if constexpr (std::is_same<T, float>::value && Q <= 3) {
    if (nb % 2 == 0) {
      if (L.nb.pdisc)
        k_spmv_nb<T, Q, D, G, true, 2><<<grid_for(threads, 256) * (nb / 2), 256, 0, s>>>(L.nb, L.ns, L.R, tc, x,
                                                                                        rhs, y, mode, nb, L.N);
      else
        k_spmv_nb<T, Q, D, G, false, 2><<<grid_for(threads, 256) * (nb / 2), 256, 0, s>>>(L.nb, L.ns, L.R, tc, x,
                                                                                         rhs, y, mode, nb, L.N);
      return;
    }
  }
  if (L.nb.pdisc) // broken pressure space
    k_spmv_nb<T, Q, D, G, true><<<grid_for(threads, 256) * nb, 256, 0, s>>>(L.nb, L.ns, L.R, tc, x, rhs, y, mode,
                                                                            nb, L.N);
  else
    k_spmv_nb<T, Q, D, G><<<grid_for(threads, 256) * nb, 256, 0, s>>>(L.nb, L.ns, L.R, tc, x, rhs, y, mode, nb,
                                                                      L.N);
}

template <typename T, int Q, int D>
void launch_spmv_qd(cudaStream_t s, const DLevel<T> &L, const TimeCoef<T> &tc, const T *x, const T *rhs, T *y,
                    int mode, int nb, int nsm) {
  if (spmv_wide_lanes(L, nsm))
    launch_spmv_qdg<T, Q, D, 32>(s, L, tc, x, rhs, y, mode, nb);
  else
    launch_spmv_qdg<T, Q, D, SpmvLanes<T, D>::G>(s, L, tc, x, rhs, y, mode, nb);
}

template <typename T, int Q>
void launch_spmv_q(cudaStream_t s, int d, const DLevel<T> &L, const TimeCoef<T> &tc, const T *x, const T *rhs,
                   T *y, int mode, int nb, int nsm) {
  if (d == 2)
    launch_spmv_qd<T, Q, 2>(s, L, tc, x, rhs, y, mode, nb, nsm);
  else
    launch_spmv_qd<T, Q, 3>(s, L, tc, x, rhs, y, mode, nb, nsm);
}

// algorithmic bytes of one Kronecker SpMV: the node-block operator once, x and y
// (and rhs) once
template <typename T>
double spmv_bytes(const DLevel<T> &L, int q, int mode) {
  return L.nb_bytes + (double)q * L.ns * sizeof(T) * (mode ? 3 : 2);
}

// nb > 1: nb columns of x, rhs, y with column stride L.N
template <int Q, int D>
void launch_mf_qd(stfem_h h, const DLevel<float> &L, const TimeCoef<float> &tc, const float *x, const float *rhs,
                  float *y, int mode, float *scratch) {
  MfDev A = L.mf;
  if (scratch) A.scratch = scratch;
  const size_t smem = (size_t)MF_CELLS * Q * (2 * A.du + A.np) * sizeof(float);
  const long ntile = (A.ncell + MF_CELLS - 1) / MF_CELLS;
  const int per_sm = std::max(1, std::min(16, (int)((227u * 1024u) / smem)));
  const long tiles = std::min<long>(ntile, std::max<long>(1, (long)h->nsm * per_sm / MF_PARTS));
  k_mf_cells<Q, D><<<(unsigned)(tiles * MF_PARTS), 32 * MF_WARPS, smem, h->stream>>>(A, tc, x);
  const long nnode = A.R / D + A.S;
  k_mf_gather<Q, D><<<grid_for((long)Q * nnode, 256), 256, 0, h->stream>>>(A, rhs, y, mode);
}

template <int Q>
void launch_mf_q(stfem_h h, const DLevel<float> &L, const TimeCoef<float> &tc, const float *x, const float *rhs,
                 float *y, int mode, float *scratch) {
  if (L.mf.d == 2)
    launch_mf_qd<Q, 2>(h, L, tc, x, rhs, y, mode, scratch);
  else
    launch_mf_qd<Q, 3>(h, L, tc, x, rhs, y, mode, scratch);
}

// y = A x (mode 0) or rhs - A x (mode 1) on a level with the matrix-free form
// (scratch: the per-cell results, nullptr = the level's own buffer)
void launch_mf(stfem_h h, const DLevel<float> &L, const TimeCoef<float> &tc, const float *x, const float *rhs,
               float *y, int mode, float *scratch = nullptr) {
  Launch G_(h, STFEM_KCLASS_SPMV, L.mf_bytes + (double)tc.q * L.ns * sizeof(float) * (mode ? 3 : 2), L.mf_flops);
  switch (tc.q) {
  case 1: launch_mf_q<1>(h, L, tc, x, rhs, y, mode, scratch); break;
  case 2: launch_mf_q<2>(h, L, tc, x, rhs, y, mode, scratch); break;
  case 3: launch_mf_q<3>(h, L, tc, x, rhs, y, mode, scratch); break;
  case 4: launch_mf_q<4>(h, L, tc, x, rhs, y, mode, scratch); break;
  default: launch_mf_q<5>(h, L, tc, x, rhs, y, mode, scratch); break;
  }
}

// floats of per-cell results the matrix-free form of a level needs
template <typename T>
size_t mf_scratch_floats(const DLevel<T> &L, int q) {
  if (!L.use_mf) return 0;
  return (size_t)L.mf.n[0] * L.mf.n[1] * L.mf.n[2] * q * (2 * L.mf.du + L.mf.np);
}

// mf_scratch: per-cell results of the matrix-free form (nullptr = the level's)
template <typename T>
void launch_spmv(stfem_h h, const DLevel<T> &L, const TimeCoef<T> &tc, const T *x, const T *rhs, T *y,
                 int mode, int nb = 1, T *mf_scratch = nullptr) {
  if constexpr (std::is_same<T, float>::value) {
    if (L.use_mf) {
      for (int c = 0; c < nb; ++c)
        launch_mf(h, L, tc, x + (long)c * L.N, rhs ? rhs + (long)c * L.N : nullptr, y + (long)c * L.N, mode,
                  mf_scratch);
      return;
    }
  }
  Launch G_(h, STFEM_KCLASS_SPMV, L.nb_bytes + (spmv_bytes(L, tc.q, mode) - L.nb_bytes) * nb,
            L.nb_flops * tc.q * nb);
  cudaStream_t s = h->stream;
  const int d = h->dim;
  const int nsm = h->nsm;
  switch (tc.q) {
  case 1: launch_spmv_q<T, 1>(s, d, L, tc, x, rhs, y, mode, nb, nsm); break;
  case 2: launch_spmv_q<T, 2>(s, d, L, tc, x, rhs, y, mode, nb, nsm); break;
  case 3: launch_spmv_q<T, 3>(s, d, L, tc, x, rhs, y, mode, nb, nsm); break;
  case 4: launch_spmv_q<T, 4>(s, d, L, tc, x, rhs, y, mode, nb, nsm); break;
  default: launch_spmv_q<T, 5>(s, d, L, tc, x, rhs, y, mode, nb, nsm); break;
  }
}

template <int Q, int D>
void launch_spmv_df_qd(cudaStream_t s, const DLevel<double> &L, const TimeCoef<double> &tc, const float *x,
                       double *y, int nb) {
  constexpr int G = D == 3 ? 8 : 4;
  const long threads = (L.nb.nu + L.nb.np) * G;
  TimeCoefDF td{};
  td.q = tc.q;
  auto pair = [](double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  };
  for (int i = 0; i < tc.q * tc.q; ++i) td.Dt[i] = pair(tc.Dt[i]);
  for (int b = 0; b < tc.q; ++b) {
    td.W[b] = pair(tc.W[b]);
    td.mW[b] = pair(-tc.W[b]);
  }
  if (L.nbdf.pdisc) // broken pressure space
    k_spmv_df<Q, D, G, true><<<grid_for(threads, 256) * nb, 256, 0, s>>>(L.nbdf, L.ns, L.R, td, x, y, nb, L.N);
  else
    k_spmv_df<Q, D, G><<<grid_for(threads, 256) * nb, 256, 0, s>>>(L.nbdf, L.ns, L.R, td, x, y, nb, L.N);
}

// y = A x on the finest FP64 level in double-float arithmetic, x FP32 (nb
// columns, stride L.N): the FGMRES operator of the MIXED mode
void launch_spmv_df(stfem_h h, const DLevel<double> &L, const TimeCoef<double> &tc, const float *x, double *y,
                    int nb = 1) {
  Launch G_(h, STFEM_KCLASS_SPMV, L.nb_bytes + (double)tc.q * L.ns * 12.0 * nb, L.nb_flops * tc.q * nb);
  cudaStream_t s = h->stream;
#define STFEM_DF_Q(Q)                                                                                  \
  if (h->dim == 2)                                                                                     \
    launch_spmv_df_qd<Q, 2>(s, L, tc, x, y, nb);                                                       \
  else                                                                                                 \
    launch_spmv_df_qd<Q, 3>(s, L, tc, x, y, nb);
  switch (tc.q) {
  case 1: STFEM_DF_Q(1) break;
  case 2: STFEM_DF_Q(2) break;
  case 3: STFEM_DF_Q(3) break;
  case 4: STFEM_DF_Q(4) break;
  default: STFEM_DF_Q(5) break;
  }
#undef STFEM_DF_Q
}

// Node-block arrays of a level in box order, decoded from the spatial system
// CSR (whose blocks have the structure of Eq. 4.7).  Every entry must lie in
// the node's neighbour box (checked); box positions without an entry are
// stored as zeros.
struct NodeBlockHost {
  long nu = 0, np = 0;
  std::vector<int> uu_ptr, up_ptr, pu_ptr, pp_ptr;
  stfem::hvec<double> uu_m, uu_k, up_c, pu_c, pp_m, pp_b;
  // broken pressure space: the "pressure nodes" are the pnl dofs of each cell;
  // up_c runs over the cells holding a displacement node (x fastest) times
  // pnl, pu_c over the (r+1)^d nodes of the dof's cell, pp_* over 2d+1 cell
  // slots (own cell, then the lower and upper neighbour along each axis; a
  // missing neighbour keeps zeros) times pnl
  bool pdisc = false;
  int pnl = 0;
};

struct HostBox {
  int lo[3], ext[3];
  long size;
};

static HostBox host_box(const int *a, int m_row, int m_col, const int *ncell, int dim) {
  HostBox b;
  b.size = 1;
  for (int i = 0; i < 3; ++i) {
    if (i < dim) {
      int clo, chi;
      stfem::cells_of(a[i], m_row, ncell[i], &clo, &chi);
      b.lo[i] = m_col * clo;
      b.ext[i] = m_col * (chi + 1) - b.lo[i] + 1;
    } else {
      b.lo[i] = 0;
      b.ext[i] = 1;
    }
    b.size *= b.ext[i];
  }
  return b;
}

// position of lattice node j (flat index in `dims`) in box b, or -1
static long box_pos(const HostBox &b, long j, const int *dims, int dim) {
  long pos = 0, stride = 1;
  for (int i = 0; i < 3; ++i) {
    int c = 0;
    if (i < dim) {
      c = (int)(j % dims[i]);
      j /= dims[i];
    }
    const int o = c - b.lo[i];
    if (o < 0 || o >= b.ext[i]) return -1;
    pos += o * stride;
    stride *= b.ext[i];
  }
  return pos;
}

static void coords_of(long idx, const int *dims, int dim, int *a) {
  for (int i = 0; i < 3; ++i) {
    if (i < dim) {
      a[i] = (int)(idx % dims[i]);
      idx /= dims[i];
    } else {
      a[i] = 0;
    }
  }
}

// Cells holding lattice node a of degree m: a box of cells, as a HostBox
// over the cell grid.
static HostBox cell_box(const int *a, int m, const int *ncell, int dim) {
  HostBox b;
  b.size = 1;
  for (int i = 0; i < 3; ++i) {
    if (i < dim) {
      int clo, chi;
      stfem::cells_of(a[i], m, ncell[i], &clo, &chi);
      b.lo[i] = clo;
      b.ext[i] = chi - clo + 1;
    } else {
      b.lo[i] = 0;
      b.ext[i] = 1;
    }
    b.size *= b.ext[i];
  }
  return b;
}

int node_block(const stfem::Level &L, int d, NodeBlockHost *out, std::string *err) {
  NodeBlockHost &H = *out;
  const long R = L.R, S = L.S, nu = R / d, np = S;
  const int r = L.r;
  const bool b1 = L.form == STFEM_FORM_PROBLEM_B_1;
  const bool disc = L.pdisc;
  const int pnl = L.pnloc;
  int nuloc = 1;
  for (int i = 0; i < d; ++i) nuloc *= r + 1;
  const int *ud = L.U.dims, *pd = L.P.dims, *nc = L.box.n;
  H.nu = nu;
  H.np = np;
  H.pdisc = disc;
  H.pnl = pnl;
  H.uu_ptr.assign(nu + 1, 0);
  H.up_ptr.assign(nu + 1, 0);
  H.pu_ptr.assign(np + 1, 0);
  H.pp_ptr.assign(np + 1, 0);
  // sizes per node (threaded), then the offsets
#pragma omp parallel for schedule(static)
  for (long I = 0; I < nu; ++I) {
    int a[3];
    coords_of(I, ud, d, a);
    H.uu_ptr[I + 1] = (int)host_box(a, r, r, nc, d).size;
    H.up_ptr[I + 1] = (int)(disc ? cell_box(a, r, nc, d).size * pnl : host_box(a, r, r - 1, nc, d).size);
  }
#pragma omp parallel for schedule(static)
  for (long sI = 0; sI < np; ++sI) {
    if (disc) {
      H.pu_ptr[sI + 1] = nuloc;
      H.pp_ptr[sI + 1] = (2 * d + 1) * pnl;
      continue;
    }
    int a[3];
    coords_of(sI, pd, d, a);
    H.pu_ptr[sI + 1] = (int)host_box(a, r - 1, r, nc, d).size;
    H.pp_ptr[sI + 1] = (int)host_box(a, r - 1, r - 1, nc, d).size;
  }
  for (long I = 0; I < nu; ++I) {
    H.uu_ptr[I + 1] += H.uu_ptr[I];
    H.up_ptr[I + 1] += H.up_ptr[I];
  }
  for (long sI = 0; sI < np; ++sI) {
    H.pu_ptr[sI + 1] += H.pu_ptr[sI];
    H.pp_ptr[sI + 1] += H.pp_ptr[sI];
  }
  auto zeros = [](stfem::hvec<double> &v, size_t n) {
    v.resize(n);
    double *p = v.data();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)n; ++i) p[i] = 0.0;
  };
  zeros(H.uu_m, H.uu_ptr[nu]);
  zeros(H.uu_k, (size_t)H.uu_ptr[nu] * d * d);
  zeros(H.up_c, (size_t)H.up_ptr[nu] * d);
  zeros(H.pu_c, (size_t)H.pu_ptr[np] * d);
  zeros(H.pp_m, H.pp_ptr[np]);
  zeros(H.pp_b, H.pp_ptr[np]);
  double scale = 0.0;
  const long nnz = (long)L.v1.size();
#pragma omp parallel for schedule(static) reduction(max : scale)
  for (long e = 0; e < nnz; ++e) scale = std::max(scale, std::max(std::fabs(L.v1[e]), std::fabs(L.v2[e])));
  const double tol = 1e-12 * scale;
  // the nodes are independent (each writes its own ranges); the first
  // structure violation found is reported
  std::atomic<const char *> fault(nullptr);
  auto node_u = [&](long I) -> const char * {
    int a[3];
    coords_of(I, ud, d, a);
    const HostBox bu = host_box(a, r, r, nc, d);
    const HostBox bp = disc ? HostBox{} : host_box(a, r, r - 1, nc, d), cb = disc ? cell_box(a, r, nc, d) : HostBox{};
    for (int c = 0; c < d; ++c) {
      // u-equation row (I, c): V block -rho M (W), U block rho M (Dt), same component
      const long ru = I * d + c;
      for (int e = L.rowptr[ru]; e < L.rowptr[ru + 1]; ++e) {
        const long col = L.col[e];
        if (col >= 2 * R) {
          if (std::fabs(L.v1[e]) > tol || std::fabs(L.v2[e]) > tol) return "u-equation couples to P";
          continue;
        }
        const long blk = col / R, rem = col % R, J = rem / d;
        const long pos = box_pos(bu, J, ud, d);
        if (pos < 0 || rem % d != c) return "u-equation entry outside the box";
        const size_t at = (size_t)H.uu_ptr[I] + pos;
        if (blk == 1) {
          if (c == 0) H.uu_m[at] = L.v1[e];
          else if (std::fabs(L.v1[e] - H.uu_m[at]) > tol) return "u-equation mass differs between components";
          if (std::fabs(L.v2[e]) > tol) return "u-equation U block has a W part";
        } else if (std::fabs(L.v1[e]) > tol) {
          return "u-equation V block has a Dt part";
        }
      }
    }
    for (int c = 0; c < d; ++c) {
      const long ru = I * d + c;
      for (int e = L.rowptr[ru]; e < L.rowptr[ru + 1]; ++e) {
        const long col = L.col[e];
        if (col < R) {
          const long pos = box_pos(bu, col / d, ud, d);
          if (pos < 0) return "u-equation V entry outside the box";
          const size_t at = (size_t)H.uu_ptr[I] + pos;
          if (std::fabs(L.v2[e] + H.uu_m[at]) > tol) return "u-equation V block is not -rho M";
        }
      }
      // v-equation row (I, c)
      const long rv = R + I * d + c;
      for (int e = L.rowptr[rv]; e < L.rowptr[rv + 1]; ++e) {
        const long col = L.col[e];
        if (col < R) {
          const long pos = box_pos(bu, col / d, ud, d);
          if (pos < 0 || col % d != c) return "v-equation V entry outside the box";
          if (std::fabs(L.v1[e] - H.uu_m[(size_t)H.uu_ptr[I] + pos]) > tol || std::fabs(L.v2[e]) > tol)
            return "v-equation V block is not rho M";
        } else if (col < 2 * R) {
          const long pos = box_pos(bu, (col - R) / d, ud, d);
          if (pos < 0 || std::fabs(L.v1[e]) > tol) return "elasticity entry outside the box";
          H.uu_k[((size_t)H.uu_ptr[I] + pos) * d * d + c * d + (col - R) % d] = L.v2[e];
        } else if (disc) {
          const long cell = (col - 2 * R) / pnl, sl = (col - 2 * R) % pnl;
          const long pos = box_pos(cb, cell, nc, d);
          if (pos < 0 || std::fabs(L.v1[e]) > tol) return "coupling entry outside the cells of the node";
          H.up_c[((size_t)H.up_ptr[I] + pos * pnl + sl) * d + c] = L.v2[e];
        } else {
          const long pos = box_pos(bp, col - 2 * R, pd, d);
          if (pos < 0 || std::fabs(L.v1[e]) > tol) return "coupling entry outside the box";
          H.up_c[((size_t)H.up_ptr[I] + pos) * d + c] = L.v2[e];
        }
      }
    }
    return nullptr;
  };
  auto node_p = [&](long sI) -> const char * {
    const long rp = 2 * R + sI;
    if (disc) {
      // broken pressure dof of cell `cell`
      const long cell = sI / pnl;
      int cm[3];
      coords_of(cell, nc, d, cm);
      for (int e = L.rowptr[rp]; e < L.rowptr[rp + 1]; ++e) {
        const long col = L.col[e];
        if ((!b1 && col < R) || (b1 && col >= R && col < 2 * R)) {
          const long rem = b1 ? col - R : col, J = rem / d;
          int aj[3];
          coords_of(J, ud, d, aj);
          int j = 0, stride = 1;
          bool in = true;
          for (int i = 0; i < d; ++i) {
            const int o = aj[i] - r * cm[i];
            in = in && o >= 0 && o <= r;
            j += o * stride;
            stride *= r + 1;
          }
          if (!in || std::fabs(b1 ? L.v2[e] : L.v1[e]) > tol) return "p-equation displacement entry outside its cell";
          H.pu_c[((size_t)H.pu_ptr[sI] + j) * d + rem % d] = b1 ? L.v1[e] : L.v2[e];
        } else if (col >= 2 * R) {
          const long cell2 = (col - 2 * R) / pnl, t = (col - 2 * R) % pnl;
          int c2[3];
          coords_of(cell2, nc, d, c2);
          int slot = -1, diff = 0;
          for (int i = 0; i < d; ++i) diff += std::abs(c2[i] - cm[i]);
          if (diff == 0) slot = 0;
          else if (diff == 1)
            for (int i = 0; i < d; ++i)
              if (c2[i] != cm[i]) slot = 1 + 2 * i + (c2[i] > cm[i] ? 1 : 0);
          if (slot < 0) return "p-equation pressure entry outside the face neighbours";
          const size_t at = (size_t)H.pp_ptr[sI] + (size_t)slot * pnl + t;
          H.pp_m[at] = L.v1[e];
          H.pp_b[at] = L.v2[e];
        } else if (std::fabs(L.v1[e]) > tol || std::fabs(L.v2[e]) > tol) {
          return b1 ? "p-equation couples to V" : "p-equation couples to U";
        }
      }
      return nullptr;
    }
    int a[3];
    coords_of(sI, pd, d, a);
    const HostBox bu = host_box(a, r - 1, r, nc, d), bp = host_box(a, r - 1, r - 1, nc, d);
    for (int e = L.rowptr[rp]; e < L.rowptr[rp + 1]; ++e) {
      const long col = L.col[e];
      if (!b1 && col < R) { // Problem 3.1: -C on V through W
        const long pos = box_pos(bu, col / d, ud, d);
        if (pos < 0 || std::fabs(L.v1[e]) > tol) return "p-equation V entry outside the box";
        H.pu_c[((size_t)H.pu_ptr[sI] + pos) * d + col % d] = L.v2[e];
      } else if (b1 && col >= R && col < 2 * R) { // Problem B.1: -C on U through Dt
        const long pos = box_pos(bu, (col - R) / d, ud, d);
        if (pos < 0 || std::fabs(L.v2[e]) > tol) return "p-equation U entry outside the box";
        H.pu_c[((size_t)H.pu_ptr[sI] + pos) * d + (col - R) % d] = L.v1[e];
      } else if (col >= 2 * R) {
        const long pos = box_pos(bp, col - 2 * R, pd, d);
        if (pos < 0) return "p-equation P entry outside the box";
        H.pp_m[(size_t)H.pp_ptr[sI] + pos] = L.v1[e];
        H.pp_b[(size_t)H.pp_ptr[sI] + pos] = L.v2[e];
      } else if (std::fabs(L.v1[e]) > tol || std::fabs(L.v2[e]) > tol) {
        return b1 ? "p-equation couples to V" : "p-equation couples to U";
      }
    }
    return nullptr;
  };
#pragma omp parallel for schedule(dynamic, 256)
  for (long I = 0; I < nu; ++I) {
    if (fault.load(std::memory_order_relaxed)) continue;
    const char *f = node_u(I);
    const char *none = nullptr;
    if (f) fault.compare_exchange_strong(none, f);
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (long sI = 0; sI < np; ++sI) {
    if (fault.load(std::memory_order_relaxed)) continue;
    const char *f = node_p(sI);
    const char *none = nullptr;
    if (f) fault.compare_exchange_strong(none, f);
  }
  if (const char *f = fault.load()) {
    *err = std::string("level operator does not have the expected block/box structure: ") + f;
    return STFEM_ERR_STATE;
  }
  return 0;
}

// Host model of the node-block product y = (Dt (x) S1 + W (x) S2) x of
// k_spmv_nb on the arrays node_block builds (FP64, one node after another),
// with the kernels' own index helpers (node_box, box_node, lattice_coords,
// disc_*): a CPU check of the layout and of the kernels' address arithmetic,
// for either pressure space.
static void block_apply_host(const NodeBlockHost &H, const stfem::Level &L, int d, int q, const double *Dt,
                             const double *W, const double *x, double *y) {
  const long R = L.R, ns = L.ns, nu = H.nu;
  const int r = L.r, pnl = H.pnl;
  const bool b1 = L.form == STFEM_FORM_PROBLEM_B_1;
  const int *ud = L.U.dims, *pd = L.P.dims, *nc = L.box.n;
  int a[3];
  for (long I = 0; I < nu; ++I) {
    lattice_coords(I, ud, d, a);
    const Box3 bu = node_box(a, r, r, nc, d);
    const Box3 bp = H.pdisc ? disc_cell_box(a, r, nc, d) : node_box(a, r, r - 1, nc, d);
    // per time node: rho M U, rho M V, K U, C^T P, each d components
    std::vector<double> mu(q * d, 0.0), mv(q * d, 0.0), ku(q * d, 0.0), cp(q * d, 0.0);
    for (int e = H.uu_ptr[I]; e < H.uu_ptr[I + 1]; ++e) {
      const long J = box_node(bu, e - H.uu_ptr[I], ud);
      for (int t = 0; t < q; ++t)
        for (int c = 0; c < d; ++c) {
          mu[t * d + c] += H.uu_m[e] * x[t * ns + R + J * d + c];
          mv[t * d + c] += H.uu_m[e] * x[t * ns + J * d + c];
          for (int c2 = 0; c2 < d; ++c2) ku[t * d + c] += H.uu_k[((size_t)e * d + c) * d + c2] * x[t * ns + R + J * d + c2];
        }
    }
    for (int e = H.up_ptr[I]; e < H.up_ptr[I + 1]; ++e) {
      const int k = e - H.up_ptr[I];
      const long sI = H.pdisc ? box_node(bp, k / pnl, nc) * pnl + k % pnl : box_node(bp, k, pd);
      for (int t = 0; t < q; ++t)
        for (int c = 0; c < d; ++c) cp[t * d + c] += H.up_c[(size_t)e * d + c] * x[t * ns + 2 * R + sI];
    }
    for (int b = 0; b < q; ++b)
      for (int c = 0; c < d; ++c) {
        double vu = 0.0, vv = 0.0;
        for (int t = 0; t < q; ++t) {
          vu += Dt[b * q + t] * mu[t * d + c];
          vv += Dt[b * q + t] * mv[t * d + c];
        }
        y[b * ns + I * d + c] = vu - W[b] * mv[b * d + c];
        y[b * ns + R + I * d + c] = vv + W[b] * (ku[b * d + c] + cp[b * d + c]);
      }
  }
  const long uoff = b1 ? R : 0;
  for (long sI = 0; sI < H.np; ++sI) {
    std::vector<double> mp(q, 0.0), bp(q, 0.0), cn(q, 0.0);
    if (H.pdisc) {
      int cm[3];
      lattice_coords(sI / pnl, nc, d, cm);
      for (int e = H.pu_ptr[sI]; e < H.pu_ptr[sI + 1]; ++e) {
        const long J = disc_cell_node(cm, e - H.pu_ptr[sI], r, ud, d);
        for (int tt = 0; tt < q; ++tt)
          for (int c = 0; c < d; ++c) cn[tt] += H.pu_c[(size_t)e * d + c] * x[tt * ns + uoff + J * d + c];
      }
      for (int e = H.pp_ptr[sI]; e < H.pp_ptr[sI + 1]; ++e) {
        const long c2 = disc_slot_cell(cm, (e - H.pp_ptr[sI]) / pnl, nc, d);
        if (c2 < 0) continue;
        const long s2 = c2 * pnl + (e - H.pp_ptr[sI]) % pnl;
        for (int tt = 0; tt < q; ++tt) {
          const double pv = x[tt * ns + 2 * R + s2];
          mp[tt] += H.pp_m[e] * pv;
          bp[tt] += H.pp_b[e] * pv;
        }
      }
    } else {
      lattice_coords(sI, pd, d, a);
      const Box3 bpx = node_box(a, r - 1, r - 1, nc, d), bux = node_box(a, r - 1, r, nc, d);
      for (int e = H.pp_ptr[sI]; e < H.pp_ptr[sI + 1]; ++e) {
        const long s2 = box_node(bpx, e - H.pp_ptr[sI], pd);
        for (int tt = 0; tt < q; ++tt) {
          mp[tt] += H.pp_m[e] * x[tt * ns + 2 * R + s2];
          bp[tt] += H.pp_b[e] * x[tt * ns + 2 * R + s2];
        }
      }
      for (int e = H.pu_ptr[sI]; e < H.pu_ptr[sI + 1]; ++e) {
        const long J = box_node(bux, e - H.pu_ptr[sI], ud);
        for (int tt = 0; tt < q; ++tt)
          for (int c = 0; c < d; ++c) cn[tt] += H.pu_c[(size_t)e * d + c] * x[tt * ns + uoff + J * d + c];
      }
    }
    for (int b = 0; b < q; ++b) {
      double v = W[b] * (bp[b] + (b1 ? 0.0 : cn[b]));
      for (int t = 0; t < q; ++t) v += Dt[b * q + t] * (mp[t] + (b1 ? cn[t] : 0.0));
      y[b * ns + 2 * R + sI] = v;
    }
  }
}

template <typename T>
int upload_level_matrix(stfem_h h, DLevel<T> &D, const stfem::Level &L, int q) {
  D.ns = L.ns;
  D.N = L.ns * q;
  D.R = L.R;
  D.S = L.S;
  NodeBlockHost H;
  std::string err;
  if (node_block(L, h->dim, &H, &err) < 0) {
    h->err = err;
    return STFEM_ERR_STATE;
  }
  const int d = h->dim;
  NodeBlockDev<T> &nb = D.nb;
  nb.nu = H.nu;
  nb.np = H.np;
  nb.r = L.r;
  nb.pcouple = L.form == STFEM_FORM_PROBLEM_B_1 ? 1 : 0;
  nb.pdisc = H.pdisc ? 1 : 0;
  nb.pnl = H.pnl;
  for (int i = 0; i < 3; ++i) {
    nb.n[i] = L.box.n[i];
    nb.udims[i] = L.U.dims[i];
    nb.pdims[i] = L.P.dims[i];
  }
  int *ip;
  T *tp;
  CKR(upload(h, &ip, H.uu_ptr)); nb.uu_ptr = ip;
  CKR(upload(h, &tp, H.uu_m)); nb.uu_m = tp;
  CKR(upload(h, &tp, H.uu_k)); nb.uu_k = tp;
  CKR(upload(h, &ip, H.up_ptr)); nb.up_ptr = ip;
  CKR(upload(h, &tp, H.up_c)); nb.up_c = tp;
  CKR(upload(h, &ip, H.pu_ptr)); nb.pu_ptr = ip;
  CKR(upload(h, &tp, H.pu_c)); nb.pu_c = tp;
  CKR(upload(h, &ip, H.pp_ptr)); nb.pp_ptr = ip;
  CKR(upload(h, &tp, H.pp_m)); nb.pp_m = tp;
  CKR(upload(h, &tp, H.pp_b)); nb.pp_b = tp;
  if (std::is_same<T, double>::value && nb.pcouple && !L.cvol.empty()) {
    // Problem B.1's previous-slab coupling: -Cvol in the layout of pu_c
    if (L.cvol.size() != H.pu_c.size()) {
      h->err = "volume coupling does not match the node-block layout";
      return STFEM_ERR_STATE;
    }
    CKR(upload(h, &tp, L.cvol));
    D.pu_cvol = tp;
  }
  const double nuu = H.uu_m.size(), nup = H.up_c.size() / d, npu = H.pu_c.size() / d, npp = H.pp_m.size();
  D.nb_bytes = (nuu * (1 + d * d) + nup * d + npu * d + npp * 2) * sizeof(T) + (2.0 * H.nu + 2.0 * H.np + 4) * 4.0;
  D.nb_flops = 2.0 * (nuu * (2 * d + d * d) + nup * d + npu * d + npp * 2);
  D.nnz = (long long)L.col.size();
  CKR(dalloc(h, &D.b, D.N));
  CKR(dalloc(h, &D.d, D.N));
  CKR(dalloc(h, &D.r, D.N));
  return 0;
}

// Float-pair copy (hi = fl32(a), lo = fl32(a - hi)) of the node-block values
// of an FP64 level, for the double-float SpMV.
// Matrix-free form of an FP32 level (continuous pressure): the unit element
// matrices in FP32, the per-cell coefficients and the per-cell result buffer.
int upload_matfree(stfem_h h, DLevel<float> &D, const stfem::Level &L) {
  const stfem::Level::Elem &E = L.elem;
  // the cell-by-cell form covers the Taylor-Hood pair with K = kappa I
  if (L.pdisc || E.nu == 0 || !L.coef.K.empty()) return 0;
  const int d = L.box.dim, nu = E.nu, np = E.np, du = nu * d;
  MfDev &A = D.mf;
  A.d = d;
  A.r = L.r;
  A.nu = nu;
  A.np = np;
  A.du = du;
  A.q = h->q;
  for (int i = 0; i < 3; ++i) {
    A.n[i] = L.box.n[i];
    A.udims[i] = L.U.dims[i];
    A.pdims[i] = L.P.dims[i];
  }
  A.R = L.R;
  A.S = L.S;
  A.ns = L.ns;
  A.pcouple = L.form == STFEM_FORM_PROBLEM_B_1 ? 1 : 0;
  A.bc_u = A.bc_p = 0;
  for (int f = 0; f < 2 * d; ++f) {
    if (L.bc.bc_u[f] == STFEM_BC_DIRICHLET) A.bc_u |= 1 << f;
    if (L.bc.bc_p[f] == STFEM_BC_DIRICHLET) A.bc_p |= 1 << f;
  }
  A.rho = (float)L.coef.rho;
  A.c0 = (float)L.coef.c0;
  float *p = nullptr;
  CKR(upload(h, &p, E.Mu)); A.Mu = p;
  CKR(upload(h, &p, E.Klam)); A.Klam = p;
  CKR(upload(h, &p, E.Kmu)); A.Kmu = p;
  CKR(upload(h, &p, E.Cv)); A.Cv = p;
  CKR(upload(h, &p, E.Bv)); A.Bv = p;
  CKR(upload(h, &p, E.Mp)); A.Mp = p;
  std::vector<double> fK((size_t)6 * 3 * du * du, 0.0), fC((size_t)6 * np * du, 0.0),
      fB((size_t)6 * 2 * np * np, 0.0);
  for (int f = 0; f < 2 * d; ++f) {
    std::copy(E.fKlam[f].begin(), E.fKlam[f].end(), fK.begin() + (size_t)f * 3 * du * du);
    std::copy(E.fKmu[f].begin(), E.fKmu[f].end(), fK.begin() + (size_t)f * 3 * du * du + (size_t)du * du);
    std::copy(E.fKpen[f].begin(), E.fKpen[f].end(), fK.begin() + (size_t)f * 3 * du * du + 2 * (size_t)du * du);
    std::copy(E.fC[f].begin(), E.fC[f].end(), fC.begin() + (size_t)f * np * du);
    std::copy(E.fB[f].begin(), E.fB[f].end(), fB.begin() + (size_t)f * 2 * np * np);
    std::copy(E.fBpen[f].begin(), E.fBpen[f].end(), fB.begin() + (size_t)f * 2 * np * np + (size_t)np * np);
  }
  CKR(upload(h, &p, fK)); A.fK = p;
  CKR(upload(h, &p, fC)); A.fC = p;
  CKR(upload(h, &p, fB)); A.fB = p;
  CKR(upload(h, &p, L.coef.lam)); A.lam = p;
  CKR(upload(h, &p, L.coef.mu)); A.mu = p;
  CKR(upload(h, &p, L.coef.kap)); A.kap = p;
  const long ncell = L.box.ncell;
  A.ncell = ncell;
  float *sc = nullptr;
  CKR(dalloc(h, &sc, (size_t)ncell * h->q * (2 * du + np)));
  A.scratch = sc;
  // algorithmic bytes beyond x and y: the per-cell results written and read
  // back, and the per-cell coefficients
  D.mf_bytes = (double)ncell * h->q * (2 * du + np) * 8.0 + ncell * 12.0;
  D.mf_flops = 2.0 * ncell * h->q * ((double)nu * nu * 2 * d + 2.0 * du * du + 2.0 * np * du + 2.0 * np * np);
  D.has_mf = true;
  return 0;
}

int upload_level_df(stfem_h h, DLevel<double> &D, const stfem::Level &L) {
  NodeBlockHost H;
  std::string err;
  if (node_block(L, h->dim, &H, &err) < 0) {
    h->err = err;
    return STFEM_ERR_STATE;
  }
  auto split = [](const stfem::hvec<double> &v) {
    stfem::hvec<float2> o(v.size());
    const long n = (long)v.size();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
      const float hi = (float)v[i];
      o[i] = make_float2(hi, (float)(v[i] - (double)hi));
    }
    return o;
  };
  NodeBlockDev<float2> &nb = D.nbdf;
  nb.nu = D.nb.nu;
  nb.np = D.nb.np;
  nb.r = D.nb.r;
  nb.pcouple = D.nb.pcouple;
  nb.pdisc = D.nb.pdisc;
  nb.pnl = D.nb.pnl;
  for (int i = 0; i < 3; ++i) {
    nb.n[i] = D.nb.n[i];
    nb.udims[i] = D.nb.udims[i];
    nb.pdims[i] = D.nb.pdims[i];
  }
  nb.uu_ptr = D.nb.uu_ptr;
  nb.up_ptr = D.nb.up_ptr;
  nb.pu_ptr = D.nb.pu_ptr;
  nb.pp_ptr = D.nb.pp_ptr;
  float2 *fp;
  CKR(upload(h, &fp, split(H.uu_m))); nb.uu_m = fp;
  CKR(upload(h, &fp, split(H.uu_k))); nb.uu_k = fp;
  CKR(upload(h, &fp, split(H.up_c))); nb.up_c = fp;
  CKR(upload(h, &fp, split(H.pu_c))); nb.pu_c = fp;
  CKR(upload(h, &fp, split(H.pp_m))); nb.pp_m = fp;
  CKR(upload(h, &fp, split(H.pp_b))); nb.pp_b = fp;
  D.has_df = true;
  return 0;
}

template <typename T>
int upload_transfer(stfem_h h, DLevel<T> &D, const stfem::CSR &Pu, const stfem::CSR &Pp) {
  stfem::CSR Ru = stfem::transpose(Pu), Rp = stfem::transpose(Pp);
  CKR(upload(h, &D.Pu_p, Pu.rowptr));
  CKR(upload(h, &D.Pu_c, Pu.col));
  CKR(upload(h, &D.Pu_v, Pu.val));
  CKR(upload(h, &D.Pp_p, Pp.rowptr));
  CKR(upload(h, &D.Pp_c, Pp.col));
  CKR(upload(h, &D.Pp_v, Pp.val));
  CKR(upload(h, &D.Ru_p, Ru.rowptr));
  CKR(upload(h, &D.Ru_c, Ru.col));
  CKR(upload(h, &D.Ru_v, Ru.val));
  CKR(upload(h, &D.Rp_p, Rp.rowptr));
  CKR(upload(h, &D.Rp_c, Rp.col));
  CKR(upload(h, &D.Rp_v, Rp.val));
  // multiply-adds of one slab transfer: q time nodes x (2d copies of the Q_r
  // operator + the Q_{r-1} operator); the operator itself is read once
  D.transfer_nnz = (double)h->q * (2.0 * h->dim * Pu.col.size() + Pp.col.size());
  D.transfer_bytes = (double)(Pu.col.size() + Pp.col.size()) * (4.0 + sizeof(T));
  return 0;
}

template <typename T>
void set_diag(DLevel<T> &D, const stfem::TimeDiag &td) {
  D.dc = DiagCoef<T>{};
  D.dc.nr = td.nr;
  D.dc.nc = td.nc;
  for (size_t i = 0; i < td.Umat.size() && i < 2 * MAXQ * MAXQ; ++i) D.dc.U[i] = (T)td.Umat[i];
  for (size_t i = 0; i < td.Vmat.size() && i < 2 * MAXQ * MAXQ; ++i) D.dc.V[i] = (T)td.Vmat[i];
}

template <typename T>
int upload_patches(stfem_h h, DLevel<T> &D, const stfem::Patches &P, double omega, int update) {
  D.npatch = P.npatch;
  D.maxC = *std::max_element(P.size.begin(), P.size.end());
  D.form = P.form;
  D.maxCs = *std::max_element(P.cs.begin(), P.cs.end());
  CKR(upload(h, &D.pcs, P.cs));
  D.inv_elems = (long long)P.inv_off.back(); // stored inverse entries (host- or device-factorised)
  D.sumC = (long long)P.dofs.size();
  // algorithmic bytes of one patch-apply launch: every inverse once (C_P^2
  // entries), the dof index, the gathered residual and the result per row
  D.patch_bytes = 0.0;
  D.patch_flops = 0.0;
  for (long p = 0; p < P.npatch; ++p) {
    const double C = P.size[p];
    const double stored = (double)(P.inv_off[p + 1] - P.inv_off[p]);
    if (P.form == 1) {
      // algorithmic: the slot inverses once (Cs^2 per real slot, 2 Cs^2 per
      // complex slot; padding excluded) plus the per-row traffic
      const double Cs = P.cs[p];
      const double q = C / Cs, nr = D.dc.nr, nc = D.dc.nc;
      D.patch_bytes += (nr + 2.0 * nc) * Cs * Cs * sizeof(T) + C * (4.0 + 2.0 * sizeof(T)) + 24.0;
      D.patch_inv_bytes += (nr + 2.0 * nc) * Cs * Cs * sizeof(T);
      D.patch_flops += (2.0 * nr + 8.0 * nc) * Cs * Cs + 4.0 * q * C;
    } else {
      D.patch_bytes += C * C * sizeof(T) + C * (4.0 + 2.0 * sizeof(T)) + 24.0;
      D.patch_inv_bytes += C * C * sizeof(T);
      D.patch_flops += 2.0 * C * C;
    }
    (void)stored;
  }
  CKR(upload(h, &D.psize, P.size));
  CKR(upload(h, &D.pld, P.ld));
  CKR(upload(h, &D.pdofs, P.dofs));
  CKR(upload(h, &D.pdoff, P.dof_off));
  CKR(upload(h, &D.pioff, P.inv_off));
  if (P.inv.empty() && P.inv_off.back() > 0) {
    CKR(dalloc(h, &D.pinv, (size_t)P.inv_off.back())); // factorised on the device
  } else {
    CKR(upload(h, &D.pinv, P.inv));
  }
  CKR(dalloc(h, &D.ybuf, P.dofs.size()));
  // inverse map dof -> positions in ybuf, in patch order
  std::vector<int> cnt(D.N + 1, 0);
  for (int dof : P.dofs) cnt[dof + 1]++;
  for (long i = 0; i < D.N; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> pos(P.dofs.size());
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (size_t e = 0; e < P.dofs.size(); ++e) pos[fill[P.dofs[e]]++] = (int)e;
  std::vector<double> scale(D.N);
  for (long i = 0; i < D.N; ++i) {
    int c = cnt[i + 1] - cnt[i];
    if (c == 0) {
      h->err = "a degree of freedom belongs to no patch";
      return STFEM_ERR_STATE;
    }
    scale[i] = update == STFEM_UPDATE_OVERWRITE ? omega : omega / c;
  }
  if (update == STFEM_UPDATE_OVERWRITE) {
    // the last patch holding a dof (positions are in patch order) wins
    std::vector<int> last(D.N);
    for (long i = 0; i < D.N; ++i) last[i] = pos[cnt[i + 1] - 1];
    pos.swap(last);
    for (long i = 0; i <= D.N; ++i) cnt[i] = (int)i;
  }
  CKR(upload(h, &D.iptr, cnt));
  CKR(upload(h, &D.ipos, pos));
  CKR(upload(h, &D.scale, scale));
  return 0;
}

// Stages of the tensor-core kernel's ring: as many as fit next to the fixed
// shared memory when STFEM_TC_CTAS_PER_SM CTAs share an SM (at most 8).
static int tc_stages(size_t fixed, int ctas_per_sm = STFEM_TC_CTAS_PER_SM) {
  const size_t per_cta = (227u * 1024u) / ctas_per_sm - 1024u;
  if (fixed >= per_cta) return 0;
  return (int)std::min<size_t>(tcp::MAXSTAGES, (per_cta - fixed) / tcp::STAGE);
}

// Time-diagonal patch inverses of a level computed on the device (see
// patch_factor.cuh): the host extracts S1_P, S2_P in batches of at most
// about 1 GB, the device forms lam_a S1_P + S2_P per slot and inverts it in
// FP64 straight into the level's storage, on a lowest-priority stream of the
// setup: when factorisation CTAs retire, kernels of other handles (the
// marches of concurrent requests) get the SMs first.
template <typename T>
int factor_on_device(stfem_h h, DLevel<T> &D, const stfem::Level &L, const stfem::Patches &P,
                     const stfem::TimeDiag &td) {
  const int ns = td.nr + td.nc;
  if (D.maxCs > 512) {
    h->err = "patches too large for the device factorisation";
    return STFEM_ERR_ARG;
  }
  double *lam = nullptr, *blocks = nullptr, *scratch = nullptr;
  long long *boff = nullptr, *bad = nullptr;
  unsigned long long *next = nullptr;
  cudaStream_t fs = nullptr;
  std::vector<double> lamh(td.lam.begin(), td.lam.end());
  lamh.resize(2 * ns, 0.0);
  const long scr_stride = 2L * D.maxCs * D.maxCs;
  const long long limit = 1LL << 30;
  const int grid = (int)std::max<long long>(1, std::min<long long>(608, limit / (scr_stride * 8)));
  int rc = 0;
  do {
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (cudaStreamCreateWithPriority(&fs, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
        cudaMalloc((void **)&lam, lamh.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&scratch, (size_t)grid * scr_stride * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&bad, sizeof(long long)) != cudaSuccess ||
        cudaMalloc((void **)&next, sizeof(unsigned long long)) != cudaSuccess) {
      h->err = "device factorisation: out of memory";
      rc = STFEM_ERR_OOM;
      break;
    }
    const long long none = LLONG_MAX;
    cudaMemcpy(lam, lamh.data(), lamh.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(bad, &none, sizeof(long long), cudaMemcpyHostToDevice);
    size_t cap_blocks = 0, cap_off = 0;
    stfem::hvec<double> hb;
    std::vector<long long> ho;
    // batches of at most `limit` bytes of blocks; the host extracts batch
    // b + 1 while the device factorises batch b (the host buffers are free
    // once their copy has landed; the device buffers once the kernel is done)
    auto batch_end = [&](long b0) {
      long b1 = b0;
      long long bytes = 0;
      while (b1 < P.npatch && (b1 == b0 || bytes + 16LL * P.cs[b1] * P.cs[b1] <= limit)) {
        bytes += 16LL * P.cs[b1] * P.cs[b1];
        ++b1;
      }
      return b1;
    };
    long p0 = 0, p1 = batch_end(0);
    if (P.npatch > 0) stfem::extract_patch_blocks(L, P, h->q, p0, p1, &hb, &ho);
    while (p0 < P.npatch && rc == 0) {
      if (hb.size() > cap_blocks) {
        if (blocks) cudaFree(blocks);
        blocks = nullptr;
        if (cudaMalloc((void **)&blocks, hb.size() * sizeof(double)) != cudaSuccess) {
          h->err = "device factorisation: out of memory";
          rc = STFEM_ERR_OOM;
          break;
        }
        cap_blocks = hb.size();
      }
      if (ho.size() > cap_off) {
        if (boff) cudaFree(boff);
        boff = nullptr;
        if (cudaMalloc((void **)&boff, ho.size() * sizeof(long long)) != cudaSuccess) {
          h->err = "device factorisation: out of memory";
          rc = STFEM_ERR_OOM;
          break;
        }
        cap_off = ho.size();
      }
      // cudaMemcpy from pageable memory may return before its DMA has landed;
      // it is ordered only with the legacy stream, so wait there before the
      // factorisation stream reads the batch (and the earlier uploads), and
      // before the host buffer is refilled
      if (cudaMemcpy(blocks, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(boff, ho.data(), ho.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaStreamSynchronize(0) != cudaSuccess) {
        h->err = "device factorisation: copy failed";
        rc = STFEM_ERR_CUDA;
        break;
      }
      const long items = (p1 - p0) * ns;
      if (cudaMemsetAsync(next, 0, sizeof(unsigned long long), fs) != cudaSuccess) {
        h->err = "device factorisation: memset failed";
        rc = STFEM_ERR_CUDA;
        break;
      }
      k_patch_factor<T><<<(int)std::min<long>(grid, items), PF_THREADS, 0, fs>>>(
          p0, p1 - p0, td.nr, td.nc, lam, D.pcs, boff, blocks, D.pioff, D.pinv, scratch, scr_stride, bad, next);
      const bool launched = cudaGetLastError() == cudaSuccess;
      const long q0 = p1, q1 = q0 < P.npatch ? batch_end(q0) : q0;
      if (launched && q0 < P.npatch) stfem::extract_patch_blocks(L, P, h->q, q0, q1, &hb, &ho);
      if (!launched || cudaStreamSynchronize(fs) != cudaSuccess) {
        h->err = "device factorisation kernel failed";
        rc = STFEM_ERR_CUDA;
        break;
      }
      p0 = q0;
      p1 = q1;
    }
    if (rc == 0) {
      long long b = none;
      cudaMemcpy(&b, bad, sizeof(long long), cudaMemcpyDeviceToHost);
      if (b != none) {
        h->err = "singular patch matrix (patch " + std::to_string(b) + ")";
        rc = STFEM_ERR_SINGULAR_PATCH;
      }
    }
  } while (false);
  if (fs) cudaStreamSynchronize(fs);
  if (lam) cudaFree(lam);
  if (blocks) cudaFree(blocks);
  if (boff) cudaFree(boff);
  if (scratch) cudaFree(scratch);
  if (bad) cudaFree(bad);
  if (next) cudaFree(next);
  if (fs) cudaStreamDestroy(fs);
  return rc;
}

// Work-item lists of the tensor-core apply of a level: whole patches, and
// single M tiles (128 rows of a patch's A, the last one possibly shorter),
// each sorted by the bytes of A it streams, largest first (ties in patch and
// tile order), so that the round-robin assignment of items to CTAs starts
// every CTA on a large item.  The default shape is whole patches, with the
// deep ring on levels of at most one patch per SM.
int build_tc_items(stfem_h h, DLevel<float> &D, const stfem::Patches &P) {
  const int nr = D.dc.nr, ns = D.dc.nr + D.dc.nc;
  for (int split = 0; split < 2; ++split) {
    std::vector<std::pair<long long, int2>> it;
    for (long p = 0; p < P.npatch; ++p) {
      const int c8 = tcp::cs8(P.cs[p]), nt = (c8 + 127) / 128;
      long long kt = 0;
      for (int a = 0; a < ns; ++a) kt += tcp::kext(a, nr, c8);
      if (!split) {
        it.push_back({(long long)c8 * kt, make_int2((int)p, nt << 16)});
      } else {
        for (int t = 0; t < nt; ++t)
          it.push_back({(long long)(std::min((t + 1) * 128, c8) - t * 128) * kt, make_int2((int)p, t | ((t + 1) << 16))});
      }
    }
    std::stable_sort(it.begin(), it.end(), [](const std::pair<long long, int2> &x,
                                              const std::pair<long long, int2> &y) { return x.first > y.first; });
    std::vector<int2> v(it.size());
    for (size_t i = 0; i < it.size(); ++i) v[i] = it[i].second;
    CKR(upload(h, &D.tc_items[split], v));
    D.tc_nitem[split] = (long)v.size();
  }
  D.tc_split = 0;
  D.tc_deep = (D.npatch <= h->nsm && D.tc_nst_deep > D.tc_nst) ? 1 : 0;
  return 0;
}

// Tensor-core tiles from device-resident FP32 inverses.
int build_tc_tiles_device(stfem_h h, DLevel<float> &D, const stfem::Patches &P) {
  const int nr = D.dc.nr, nc = D.dc.nc, ns = nr + nc, nrow = nr + 2 * nc;
  const int c8max = tcp::cs8(D.maxCs);
  if (c8max * 32 > tcp::STAGE) {
    h->err = "patches too large for the tensor-core patch apply";
    return STFEM_ERR_ARG;
  }
  const size_t fixed = tcp::smem_bytes(0, D.maxCs, nrow);
  const int nst = tc_stages(fixed);
  if (nst < 2) {
    h->err = "patches too large for the tensor-core patch apply (shared memory)";
    return STFEM_ERR_ARG;
  }
  // one accumulator per slot and M tile; two CTAs per SM share its 512 columns
  const uint32_t cols = tcp::tmem_cols(ns, c8max);
  if (cols > 512u / STFEM_TC_CTAS_PER_SM) {
    h->err = "patches too large for the tensor-core patch apply (tensor memory)";
    return STFEM_ERR_ARG;
  }
  std::vector<long long> off(P.npatch + 1, 0);
  for (long p = 0; p < P.npatch; ++p) {
    const long long c8 = tcp::cs8(P.cs[p]);
    long long n = 0;
    for (int a = 0; a < ns; ++a) n += (long long)tcp::kext(a, nr, (int)c8) * c8;
    off[p + 1] = off[p] + n;
  }
  CKR(upload(h, &D.ptoff, off));
  CKR(dalloc(h, &D.ptile, (size_t)off[P.npatch]));
  k_build_tc_tiles<<<(unsigned)P.npatch, 256>>>(D.pcs, D.pioff, D.pinv, D.ptoff, D.ptile, nr, nc);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(0));
  D.tc = 1;
  D.tc_nst = nst;
  D.tc_nst_deep = tc_stages(fixed, 1);
  D.tc_cols = cols;
  return build_tc_items(h, D, P);
}

// Level work vectors with nb columns (b, d, r of N; the patch results of sumC).
template <typename T>
int ensure_columns(stfem_h h, DLevel<T> &D, int nb) {
  if (D.ncols >= nb) return 0;
  CKR(dalloc(h, &D.b, (size_t)nb * D.N));
  CKR(dalloc(h, &D.d, (size_t)nb * D.N));
  CKR(dalloc(h, &D.r, (size_t)nb * D.N));
  if (D.sumC > 0) CKR(dalloc(h, &D.ybuf, (size_t)nb * D.sumC));
  D.ncols = nb;
  return 0;
}

// Tensor-core layout of the time-diagonal inverses of an FP32 level (see
// tc_patch.cuh): per patch and slot a, A(m, k) in K blocks of 8, row groups
// of 8, K cores of 4; real slot A = Z_a, complex slot A = [Re Z_a | Im Z_a];
// rows padded to Cs8, K to Cs8 or 2 Cs8, with zeros.
int upload_tc_tiles(stfem_h h, DLevel<float> &D, const stfem::Patches &P) {
  const int nr = D.dc.nr, nc = D.dc.nc, ns = nr + nc, nrow = nr + 2 * nc;
  const int c8max = tcp::cs8(D.maxCs);
  if (c8max * 32 > tcp::STAGE) {
    h->err = "patches too large for the tensor-core patch apply";
    return STFEM_ERR_ARG;
  }
  const size_t fixed = tcp::smem_bytes(0, D.maxCs, nrow);
  const int nst = tc_stages(fixed);
  if (nst < 2) {
    h->err = "patches too large for the tensor-core patch apply (shared memory)";
    return STFEM_ERR_ARG;
  }
  // one accumulator per slot and M tile; two CTAs per SM share its 512 columns
  const uint32_t cols = tcp::tmem_cols(ns, c8max);
  if (cols > 512u / STFEM_TC_CTAS_PER_SM) {
    h->err = "patches too large for the tensor-core patch apply (tensor memory)";
    return STFEM_ERR_ARG;
  }
  std::vector<long long> off(P.npatch + 1, 0);
  for (long p = 0; p < P.npatch; ++p) {
    const long long c8 = tcp::cs8(P.cs[p]);
    long long n = 0;
    for (int a = 0; a < ns; ++a) n += (long long)tcp::kext(a, nr, (int)c8) * c8;
    off[p + 1] = off[p] + n;
  }
  std::vector<float> tile((size_t)off[P.npatch], 0.f);
  for (long p = 0; p < P.npatch; ++p) {
    const int Cs = P.cs[p], c8 = tcp::cs8(Cs);
    const int ldR = (Cs + 3) / 4 * 4, ldC = 2 * ((Cs + 1) / 2 * 2);
    const double *inv = P.inv.data() + P.inv_off[p];
    float *t = tile.data() + off[p];
    for (int a = 0; a < ns; ++a) {
      const int K = tcp::kext(a, nr, c8);
      auto at = [&](int m, int k) -> float & {
        return t[(size_t)(k / 8) * c8 * 8 + ((m / 8) * 2 + (k % 8) / 4) * 32 + (m % 8) * 4 + (k % 4)];
      };
      if (a < nr) {
        const double *z = inv + (size_t)a * Cs * ldR;
        for (int j = 0; j < Cs; ++j)
          for (int m = 0; m < Cs; ++m) at(m, j) = (float)z[(size_t)j * ldR + m];
      } else {
        const double *z = inv + (size_t)nr * Cs * ldR + (size_t)(a - nr) * Cs * ldC;
        for (int j = 0; j < Cs; ++j)
          for (int m = 0; m < Cs; ++m) {
            at(m, j) = (float)z[(size_t)j * ldC + 2 * m];
            at(m, c8 + j) = (float)z[(size_t)j * ldC + 2 * m + 1];
          }
      }
      t += (size_t)K * c8;
    }
  }
  CKR(upload(h, &D.ptoff, off));
  CKR(upload(h, &D.ptile, tile));
  D.tc = 1;
  D.tc_nst = nst;
  D.tc_nst_deep = tc_stages(fixed, 1);
  D.tc_cols = cols;
  return build_tc_items(h, D, P);
}

// ---------------------------------------------------------------- V-cycle
template <typename T>
std::vector<DLevel<T>> &levels(stfem_h h);
template <>
std::vector<DLevel<double>> &levels<double>(stfem_h h) {
  return h->L64;
}
template <>
std::vector<DLevel<float>> &levels<float>(stfem_h h) {
  return h->L32;
}

// Launch shape of the patch apply: RT row threads cover the largest patch
// (VEC rows each, or the slot rows of the time-diagonal form); J column groups
// per patch when the level has too few patches to keep the 152 SMs streaming
// (about 2^18 resident threads).
template <typename T, int Q>
void launch_patch_diag_q(cudaStream_t s, DLevel<T> &L, int RT, int J, size_t smem, const T *res, T *y) {
  const unsigned grid = (unsigned)L.npatch;
  switch (J) {
  case 1: k_patch_apply_diag<T, 1, Q><<<grid, RT, smem, s>>>(L.pcs, L.pdoff, L.pdofs, L.pioff, L.pinv, res, y, L.dc, L.maxCs); break;
  case 2: k_patch_apply_diag<T, 2, Q><<<grid, RT * 2, smem, s>>>(L.pcs, L.pdoff, L.pdofs, L.pioff, L.pinv, res, y, L.dc, L.maxCs); break;
  case 4: k_patch_apply_diag<T, 4, Q><<<grid, RT * 4, smem, s>>>(L.pcs, L.pdoff, L.pdofs, L.pioff, L.pinv, res, y, L.dc, L.maxCs); break;
  default: k_patch_apply_diag<T, 8, Q><<<grid, RT * 8, smem, s>>>(L.pcs, L.pdoff, L.pdofs, L.pioff, L.pinv, res, y, L.dc, L.maxCs); break;
  }
}

// Threads per CTA of k_patch_apply_wide; a level takes that kernel when it has
// at most STFEM_WIDE_MAX_PATCHES_PER_SM patches per multiprocessor (a fixed
// rule, not a timing, so that the arithmetic of a level never depends on the
// run) and each slot's row groups fit one CTA.
constexpr int WIDE_THREADS = 512;
#ifndef STFEM_WIDE_MAX_PATCHES_PER_SM
#define STFEM_WIDE_MAX_PATCHES_PER_SM 1
#endif

template <typename T>
size_t wide_smem(const DLevel<T> &L, int q) {
  return ((size_t)(q + 2) * L.maxCs + (size_t)WIDE_THREADS * Vec16<T>::n) * sizeof(T);
}

// the level's patches fit k_patch_apply_wide (time-diagonal form, FP32 or
// FP64 CUDA cores, every slot's row groups in one CTA)
template <typename T>
bool wide_possible(const DLevel<T> &L) {
  constexpr int CR = Vec16<T>::n / 2;
  return L.form == 1 && !L.tc && L.npatch > 0 && (L.maxCs + CR - 1) / CR <= WIDE_THREADS &&
         wide_smem(L, MAXQ) <= 227u * 1024u;
}

// kernel choice of a level: STFEM_PATCH_KERNEL_AUTO takes the wide kernel for
// levels with few patches, the streaming kernel for the others
template <typename T>
bool wide_chosen(const DLevel<T> &L, int nsm, int choice) {
  if (!wide_possible(L) || choice == STFEM_PATCH_KERNEL_STREAM) return false;
  return choice == STFEM_PATCH_KERNEL_WIDE || L.npatch <= (long)STFEM_WIDE_MAX_PATCHES_PER_SM * nsm;
}

// Shape of the streaming time-diagonal patch apply: one consumer thread per
// row block of the largest patch (rounded to warps) plus a producer warp;
// shared memory = stages + the per-patch vectors; as many CTAs per SM as
// shared memory allows (at most 3), at most one CTA per patch.
// Ring shape (measured on GB300 with both bench workloads): 2D patches (few
// consumer warps per CTA) run best with 2 stages and up to 5 CTAs per SM,
// 3D patches with 4 stages and up to 3.
template <typename T>
void stream_shape(stfem_h h, const DLevel<T> &L, int *threads, size_t *smem, int *grid, int *nst) {
  const int q = h->q, dim = h->dim;
  constexpr int VEC = Vec16<T>::n;
  const int rows = L.dc.nr * ((L.maxCs + VEC - 1) / VEC) + L.dc.nc * ((L.maxCs + VEC / 2 - 1) / (VEC / 2));
  const int nwc = std::max(1, (rows + 31) / 32);
  *threads = 32 * (nwc + 1);
  *nst = dim == 2 ? 2 : 4;
  int cap = dim == 2 ? 5 : 3;
  if (L.tune_nst > 0) {
    *nst = L.tune_nst;
    cap = L.tune_cap;
  }
  *smem = (size_t)stream_header(*nst) + (size_t)(q + 2 * (L.dc.nr + 2 * L.dc.nc)) * L.maxCs * sizeof(T);
  const int per_sm = std::max(1, std::min(cap, (int)((227u * 1024u) / *smem)));
  *grid = (int)std::min<long>(L.npatch, (long)h->nsm * per_sm);
  if (h->launch_cap > 0) *grid = std::min(*grid, h->launch_cap);
}

// Appends a level's patches (input res, results y; slot results zb and
// tickets tk for the wide kernel) to a job table.
template <typename T, int MAXJ>
void add_job(PatchJobs<T, MAXJ> &J, const DLevel<T> &L, const T *res, T *y, T *zb = nullptr, int *tk = nullptr) {
  const int j = J.njobs++;
  if (j == 0) J.first[0] = 0;
  J.first[j + 1] = J.first[j] + L.npatch;
  J.pcs[j] = L.pcs;
  J.pdoff[j] = L.pdoff;
  J.pdofs[j] = L.pdofs;
  J.pioff[j] = L.pioff;
  J.pinv[j] = L.pinv;
  J.res[j] = res;
  J.y[j] = y;
  J.zbuf[j] = zb;
  J.ticket[j] = tk;
  J.dc[j] = L.dc;
}

template <typename T, int Q>
void launch_patch_stream_q(stfem_h h, DLevel<T> &L, const T *res, T *y) {
  int threads, grid, nst;
  size_t smem;
  stream_shape(h, L, &threads, &smem, &grid, &nst);
  PatchJobs<T, 1> J;
  J.njobs = 0;
  add_job(J, L, res, y);
  const int tile = L.tune_tile > 0 ? L.tune_tile : 1;
  grid = std::max(1, std::min<int>(grid, (int)((L.npatch + tile - 1) / tile)));
  k_patch_apply_stream<T, Q, 1><<<grid, threads, smem, h->stream>>>(J, L.maxCs, tile, h->dev_err, nst,
                                                                    h->wait_cycles, h->stall_copies);
}

template <typename T, int Q>
void launch_patch_wide_q(stfem_h h, DLevel<T> &L, const T *res, T *y, T *zb, int *tk) {
  const size_t smem = wide_smem<T>(L, Q);
  const int ns = L.dc.nr + L.dc.nc;
  PatchJobs<T, 1> J;
  J.njobs = 0;
  add_job(J, L, res, y, zb, tk);
  k_patch_apply_wide<T, Q, PatchJobs<T, 1>><<<(unsigned)(L.npatch * ns), WIDE_THREADS, smem, h->stream>>>(J);
}

// zb, tk: slot results and ticket counters of the wide kernel (nullptr: the
// level's own)
template <typename T>
void launch_patch_apply_to(stfem_h h, DLevel<T> &L, const T *res, T *y, T *zb = nullptr, int *tk = nullptr) {
  constexpr int VEC = Vec16<T>::n;
  if (L.form == 1 && L.wide) {
    if (!zb) zb = L.zbuf;
    if (!tk) tk = L.ticket;
    switch (h->q) {
    case 1: launch_patch_wide_q<T, 1>(h, L, res, y, zb, tk); break;
    case 2: launch_patch_wide_q<T, 2>(h, L, res, y, zb, tk); break;
    case 3: launch_patch_wide_q<T, 3>(h, L, res, y, zb, tk); break;
    case 4: launch_patch_wide_q<T, 4>(h, L, res, y, zb, tk); break;
    default: launch_patch_wide_q<T, 5>(h, L, res, y, zb, tk); break;
    }
    return;
  }
  int rows;
  if (L.form == 1)
    rows = L.dc.nr * ((L.maxCs + VEC - 1) / VEC) + L.dc.nc * ((L.maxCs + VEC / 2 - 1) / (VEC / 2));
  else
    rows = (L.maxC + VEC - 1) / VEC;
  // the dense kernel loops over row blocks, so it can cap RT; the
  // time-diagonal one needs every row block resident (checked at setup)
  const int RT = L.form == 1 ? std::max((rows + 31) / 32 * 32, 32) : std::min(std::max((rows + 31) / 32 * 32, 32), 512);
  int J = 1;
  const double target = (double)h->nsm * STFEM_PATCH_THREADS_PER_SM;
  while (J < 8 && (double)L.npatch * RT * J < target && RT * J * 2 <= 1024) J *= 2;
  size_t smem = (J > 1 ? (size_t)J * RT * VEC * sizeof(T) : 0);
  cudaStream_t s = h->stream;
  const unsigned grid = (unsigned)L.npatch;
  if (L.form == 1 && L.npatch < STFEM_STREAM_MIN_PATCHES) {
    smem += (size_t)(h->q + 2 * (L.dc.nr + 2 * L.dc.nc)) * L.maxCs * sizeof(T);
    switch (h->q) {
    case 1: launch_patch_diag_q<T, 1>(s, L, RT, J, smem, res, y); break;
    case 2: launch_patch_diag_q<T, 2>(s, L, RT, J, smem, res, y); break;
    case 3: launch_patch_diag_q<T, 3>(s, L, RT, J, smem, res, y); break;
    case 4: launch_patch_diag_q<T, 4>(s, L, RT, J, smem, res, y); break;
    default: launch_patch_diag_q<T, 5>(s, L, RT, J, smem, res, y); break;
    }
    return;
  }
  if (L.form == 1) {
    switch (h->q) {
    case 1: launch_patch_stream_q<T, 1>(h, L, res, y); break;
    case 2: launch_patch_stream_q<T, 2>(h, L, res, y); break;
    case 3: launch_patch_stream_q<T, 3>(h, L, res, y); break;
    case 4: launch_patch_stream_q<T, 4>(h, L, res, y); break;
    default: launch_patch_stream_q<T, 5>(h, L, res, y); break;
    }
    return;
  }
  smem += (size_t)L.maxC * sizeof(T);
  switch (J) {
  case 1: k_patch_apply<T, 1><<<grid, RT, smem, s>>>(L.psize, L.pdoff, L.pdofs, L.pioff, L.pld, L.pinv, res, y); break;
  case 2: k_patch_apply<T, 2><<<grid, RT * 2, smem, s>>>(L.psize, L.pdoff, L.pdofs, L.pioff, L.pld, L.pinv, res, y); break;
  case 4: k_patch_apply<T, 4><<<grid, RT * 4, smem, s>>>(L.psize, L.pdoff, L.pdofs, L.pioff, L.pld, L.pinv, res, y); break;
  default: k_patch_apply<T, 8><<<grid, RT * 8, smem, s>>>(L.psize, L.pdoff, L.pdofs, L.pioff, L.pld, L.pinv, res, y); break;
  }
}

// Opts the streaming kernels in to 227 KB of dynamic shared memory (done at
// setup, never during a graph capture).
int prepare_stream_kernels(stfem_h h) {
#define STFEM_SMEM_ATTR(T, Q)                                                                            \
  CK(cudaFuncSetAttribute(k_patch_apply_stream<T, Q, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)); \
  CK(cudaFuncSetAttribute(k_patch_apply_stream<T, Q, MAXJOBS>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                          227 * 1024))
  STFEM_SMEM_ATTR(float, 1); STFEM_SMEM_ATTR(float, 2); STFEM_SMEM_ATTR(float, 3);
  STFEM_SMEM_ATTR(float, 4); STFEM_SMEM_ATTR(float, 5);
  STFEM_SMEM_ATTR(double, 1); STFEM_SMEM_ATTR(double, 2); STFEM_SMEM_ATTR(double, 3);
  STFEM_SMEM_ATTR(double, 4); STFEM_SMEM_ATTR(double, 5);
#undef STFEM_SMEM_ATTR
#define STFEM_SMEM_ATTR_W(T, Q)                                                                          \
  CK(cudaFuncSetAttribute(k_patch_apply_wide<T, Q, PatchJobs<T, 1>>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                          227 * 1024));                                                                        \
  CK(cudaFuncSetAttribute(k_patch_apply_wide<T, Q, PatchJobs<T, MAXJOBS>>,                                     \
                          cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024))
  STFEM_SMEM_ATTR_W(float, 1); STFEM_SMEM_ATTR_W(float, 2); STFEM_SMEM_ATTR_W(float, 3);
  STFEM_SMEM_ATTR_W(float, 4); STFEM_SMEM_ATTR_W(float, 5);
  STFEM_SMEM_ATTR_W(double, 1); STFEM_SMEM_ATTR_W(double, 2); STFEM_SMEM_ATTR_W(double, 3);
  STFEM_SMEM_ATTR_W(double, 4); STFEM_SMEM_ATTR_W(double, 5);
#undef STFEM_SMEM_ATTR_W
#define STFEM_SMEM_ATTR_MF(Q)                                                                            \
  CK(cudaFuncSetAttribute(k_mf_cells<Q, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));   \
  CK(cudaFuncSetAttribute(k_mf_cells<Q, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024))
  STFEM_SMEM_ATTR_MF(1); STFEM_SMEM_ATTR_MF(2); STFEM_SMEM_ATTR_MF(3); STFEM_SMEM_ATTR_MF(4); STFEM_SMEM_ATTR_MF(5);
#undef STFEM_SMEM_ATTR_MF
  CK(cudaFuncSetAttribute(k_patch_apply_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  CK(cudaFuncSetAttribute(k_patch_apply_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  CK(cudaFuncSetAttribute(k_patch_apply_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  CK(cudaFuncSetAttribute(k_patch_apply_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  CK(cudaFuncSetAttribute(k_patch_apply_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  return 0;
}

template <typename T>
int prepare_wide(stfem_h h, DLevel<T> &L) {
  L.wide = wide_chosen(L, h->nsm, h->patch_kernel) ? 1 : 0;
  if (!L.wide || L.zbuf) return 0;
  CKR(dalloc(h, &L.zbuf, (size_t)L.sumC));
  CKR(dalloc(h, &L.ticket, (size_t)L.npatch));
  CK(cudaMemset(L.ticket, 0, (size_t)L.npatch * sizeof(int)));
  return 0;
}

// Autotuner of the streaming patch apply: times the candidate ring shapes
// (stages per CTA x CTAs per SM) and patch tiles (consecutive patches a CTA
// takes per step) on the level's own inverses and keeps the fastest.  The
// shape and the tile change only how patches are spread over CTAs, never the
// arithmetic of a patch, so results do not depend on the choice.
template <typename T>
int autotune_stream(stfem_h h, DLevel<T> &L) {
  if (L.form != 1 || L.tc || L.wide || L.npatch == 0) return 0;
  static const int cand[][3] = STREAM_SHAPE_CANDIDATES;
  cudaStream_t ts = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStream_t saved = h->stream;
  h->stream = ts;
  cudaMemsetAsync(L.r, 0, (size_t)L.N * sizeof(T), ts);
  float best = 1e30f;
  int bn = 0, bc = 0, bt = 0;
  for (const auto &c : cand) {
    L.tune_nst = c[0];
    L.tune_cap = c[1];
    L.tune_tile = c[2];
    int threads, grid, nst;
    size_t smem;
    stream_shape(h, L, &threads, &smem, &grid, &nst);
    if (smem > 227u * 1024u) continue;
    for (int w = 0; w < 2; ++w) launch_patch_apply_to<T>(h, L, L.r, L.ybuf);
    cudaEventRecord(e0, ts);
    for (int t = 0; t < 5; ++t) launch_patch_apply_to<T>(h, L, L.r, L.ybuf);
    cudaEventRecord(e1, ts);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bn = c[0];
      bc = c[1];
      bt = c[2];
    }
  }
  h->stream = saved;
  L.tune_nst = bn;
  L.tune_cap = bc;
  L.tune_tile = bt;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaStreamSynchronize(ts);
  cudaStreamDestroy(ts);
  CK(e);
  CK(cudaGetLastError());
  return 0;
}

// Row threads a patch needs: the time-diagonal kernel gives each thread one
// row block; a single CTA (no column split) holds at most 512 threads.
template <typename T>
int check_patch_shape(stfem_h h, const DLevel<T> &L) {
  constexpr int VEC = Vec16<T>::n;
  if (L.form != 1) return 0;
  const int rows = L.dc.nr * ((L.maxCs + VEC - 1) / VEC) + L.dc.nc * ((L.maxCs + VEC / 2 - 1) / (VEC / 2));
  int threads, grid, nst;
  size_t smem;
  stream_shape(h, L, &threads, &smem, &grid, &nst);
  const size_t widest_column = (size_t)2 * ((L.maxCs + 1) / 2 * 2) * sizeof(T); // complex slot column
  if (rows > 992 || smem > 227u * 1024u || widest_column > (size_t)STREAM_CHUNK) {
    h->err = "patches too large for the time-diagonal form (" + std::to_string(rows) + " row threads, " +
             std::to_string(smem) + " bytes of shared memory); use STFEM_PATCH_DENSE";
    return STFEM_ERR_ARG;
  }
  return 0;
}

// y: nb columns of sumC patch results (column stride L.sumC)
template <int Q>
void launch_patch_tc_q(stfem_h h, DLevel<float> &L, const float *res, float *y, int nb) {
  // the level's shape (autotune_tc): whole patches or single M tiles as work
  // items; the shared ring of STFEM_TC_CTAS_PER_SM CTAs per SM, or one CTA per
  // SM with the deepest ring (where a CTA's bytes in flight bound the level)
  const int split = L.tc_split, deep = L.tc_deep && L.tc_nst_deep > L.tc_nst;
  const int nst = deep ? L.tc_nst_deep : L.tc_nst;
  const long nitem = L.tc_nitem[split];
  const size_t smem = tcp::smem_bytes(nst, L.maxCs, L.dc.nr + 2 * L.dc.nc);
  int grid = (int)std::min<long>(nitem, (long)h->nsm * (deep ? 1 : STFEM_TC_CTAS_PER_SM));
  if (h->launch_cap > 0) grid = std::min(grid, h->launch_cap);
  if (grid <= 0) return;
  k_patch_apply_tc<Q><<<grid, tcp::THREADS, smem, h->stream>>>((int)nitem, L.tc_items[split], nb, L.pcs, L.pdoff,
                                                             L.pdofs, L.ptoff, L.ptile, res, L.N, y, L.sumC, L.dc,
                                                             L.maxCs, nst, L.tc_cols, h->dev_err);
}

// the tensor-core apply of a level into y (nb columns)
void launch_patch_tc(stfem_h h, DLevel<float> &L, const float *res, float *y, int nb) {
  switch (h->q) {
  case 1: launch_patch_tc_q<1>(h, L, res, y, nb); break;
  case 2: launch_patch_tc_q<2>(h, L, res, y, nb); break;
  case 3: launch_patch_tc_q<3>(h, L, res, y, nb); break;
  case 4: launch_patch_tc_q<4>(h, L, res, y, nb); break;
  default: launch_patch_tc_q<5>(h, L, res, y, nb); break;
  }
}

// nb columns: res with column stride L.N, results with column stride
// L.sumC.  Algorithmic bytes: the inverses once, the per-row traffic per
// column (the tensor-core kernel reads each inverse once for all columns;
// without it the columns are applied one after another).
// Autotuner of the tensor-core patch apply (FP32 levels of handles set up for
// several right-hand sides): times whole-patch and single-tile work items,
// each with the shared ring and (where one fits) the deeper one-CTA-per-SM
// ring, on the level's own tiles with the handle's column count, and keeps
// the fastest.  Items and rings change only how rows are spread over CTAs,
// never the arithmetic of a row, so results do not depend on the choice.
int autotune_tc(stfem_h h, DLevel<float> &L) {
  if (!L.tc || L.npatch == 0) return 0;
  const int nb = std::max(1, std::min(h->nrhs_cap, L.ncols));
  cudaStream_t ts = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStream_t saved = h->stream;
  h->stream = ts;
  cudaMemsetAsync(L.r, 0, (size_t)nb * L.N * sizeof(float), ts);
  float best = 1e30f;
  int bs = L.tc_split, bd = L.tc_deep;
  for (int split = 0; split < 2; ++split)
    for (int deep = 0; deep < 2; ++deep) {
      if (deep && L.tc_nst_deep <= L.tc_nst) continue;
      L.tc_split = split;
      L.tc_deep = deep;
      for (int w = 0; w < 2; ++w) launch_patch_tc(h, L, L.r, L.ybuf, nb);
      cudaEventRecord(e0, ts);
      for (int t = 0; t < 5; ++t) launch_patch_tc(h, L, L.r, L.ybuf, nb);
      cudaEventRecord(e1, ts);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bs = split;
        bd = deep;
      }
    }
  h->stream = saved;
  L.tc_split = bs;
  L.tc_deep = bd;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaStreamSynchronize(ts);
  cudaStreamDestroy(ts);
  CK(e);
  CK(cudaGetLastError());
  return 0;
}

template <typename T>
void launch_patch_apply(stfem_h h, DLevel<T> &L, const T *res, int nb = 1) {
  Launch G_(h, STFEM_KCLASS_PATCH_APPLY, L.patch_inv_bytes + (L.patch_bytes - L.patch_inv_bytes) * nb,
            L.patch_flops * nb);
  if constexpr (std::is_same<T, float>::value) {
    if (L.tc) {
      launch_patch_tc(h, L, res, L.ybuf, nb);
      return;
    }
  }
  for (int c = 0; c < nb; ++c) launch_patch_apply_to<T>(h, L, res + (long)c * L.N, L.ybuf + (long)c * L.sumC);
}

// nsw sweeps of Algorithm 4.1 on level l for nb columns of the level buffers
template <typename T>
void smooth(stfem_h h, int l, int nsw, bool zero_init, int nb = 1) {
  DLevel<T> &L = levels<T>(h)[l];
  const TimeCoef<T> tc = time_coef<T>(h->T, h->tau);
  cudaStream_t s = h->stream;
  for (int it = 0; it < nsw; ++it) {
    const bool zero = zero_init && it == 0;
    const T *res = L.b;
    if (!zero) {
      launch_spmv<T>(h, L, tc, L.d, L.b, L.r, 1, nb);
      res = L.r;
    }
    launch_patch_apply<T>(h, L, res, nb);
    {
      Launch G_(h, STFEM_KCLASS_UPDATE,
                ((double)L.N * (4.0 + 3.0 * sizeof(T)) + (double)L.sumC * (4.0 + sizeof(T))) * nb,
                ((double)L.sumC + 2.0 * L.N) * nb);
      k_vanka_update<T><<<grid_for(L.N, 256) * nb, 256, 0, s>>>(L.N, L.iptr, L.ipos, L.scale, L.ybuf, L.d,
                                                                zero ? 1 : 0, nb, L.sumC);
    }
  }
}

template <typename T>
void restrict_to(stfem_h h, int l, const T *rf, T *bc, int nb = 1) {
  DLevel<T> &F = levels<T>(h)[l];
  DLevel<T> &C = levels<T>(h)[l - 1];
  Launch G_(h, STFEM_KCLASS_TRANSFER, (double)(C.N + F.N) * sizeof(T) * nb + F.transfer_bytes,
            2.0 * F.transfer_nnz * nb);
  // restriction: rows of P^T are long, STFEM_RESTRICT_LANES lanes per output
  const long nu = C.R / h->dim, np = C.S, nt = (2 * nu + np) * h->q;
  constexpr int GR = STFEM_RESTRICT_LANES;
  // small coarse levels: a warp per output (fewer dependent trips per lane)
  const bool wide = nt * 32 <= (long)h->nsm * 1024;
  if (h->dim == 2) {
    if (wide)
      k_transfer<T, 2, 32><<<grid_for(nt * 32, 128) * nb, 128, 0, h->stream>>>(
          nu, np, h->q, C.ns, C.R, F.ns, F.R, F.Ru_p, F.Ru_c, F.Ru_v, F.Rp_p, F.Rp_c, F.Rp_v, rf, bc, 0, nb, F.N, C.N);
    else
      k_transfer<T, 2, GR><<<grid_for(nt * GR, 128) * nb, 128, 0, h->stream>>>(
          nu, np, h->q, C.ns, C.R, F.ns, F.R, F.Ru_p, F.Ru_c, F.Ru_v, F.Rp_p, F.Rp_c, F.Rp_v, rf, bc, 0, nb, F.N, C.N);
  } else {
    if (wide)
      k_transfer<T, 3, 32><<<grid_for(nt * 32, 128) * nb, 128, 0, h->stream>>>(
          nu, np, h->q, C.ns, C.R, F.ns, F.R, F.Ru_p, F.Ru_c, F.Ru_v, F.Rp_p, F.Rp_c, F.Rp_v, rf, bc, 0, nb, F.N, C.N);
    else
      k_transfer<T, 3, GR><<<grid_for(nt * GR, 128) * nb, 128, 0, h->stream>>>(
          nu, np, h->q, C.ns, C.R, F.ns, F.R, F.Ru_p, F.Ru_c, F.Ru_v, F.Rp_p, F.Rp_c, F.Rp_v, rf, bc, 0, nb, F.N, C.N);
  }
}

template <typename T>
void prolongate_add(stfem_h h, int l, const T *dc, T *df, int nb = 1) {
  DLevel<T> &F = levels<T>(h)[l];
  DLevel<T> &C = levels<T>(h)[l - 1];
  Launch G_(h, STFEM_KCLASS_TRANSFER, (double)(C.N + 2 * F.N) * sizeof(T) * nb + F.transfer_bytes,
            2.0 * F.transfer_nnz * nb);
  const long nu = F.R / h->dim, np = F.S, nt = (2 * nu + np) * h->q;
  constexpr int GP = STFEM_PROLONG_LANES;
  // small fine levels: 8 lanes per output (rows of P hold up to (r+1)^d entries)
  const bool wide = nt * 8 <= (long)h->nsm * 1024;
  if (h->dim == 2) {
    if (wide)
      k_transfer<T, 2, 8><<<grid_for(nt * 8, 128) * nb, 128, 0, h->stream>>>(
          nu, np, h->q, F.ns, F.R, C.ns, C.R, F.Pu_p, F.Pu_c, F.Pu_v, F.Pp_p, F.Pp_c, F.Pp_v, dc, df, 1, nb, C.N, F.N);
    else
      k_transfer<T, 2, GP><<<grid_for(nt * GP, 128) * nb, 128, 0, h->stream>>>(
          nu, np, h->q, F.ns, F.R, C.ns, C.R, F.Pu_p, F.Pu_c, F.Pu_v, F.Pp_p, F.Pp_c, F.Pp_v, dc, df, 1, nb, C.N, F.N);
  } else {
    if (wide)
      k_transfer<T, 3, 8><<<grid_for(nt * 8, 128) * nb, 128, 0, h->stream>>>(
          nu, np, h->q, F.ns, F.R, C.ns, C.R, F.Pu_p, F.Pu_c, F.Pu_v, F.Pp_p, F.Pp_c, F.Pp_v, dc, df, 1, nb, C.N, F.N);
    else
      k_transfer<T, 3, GP><<<grid_for(nt * GP, 128) * nb, 128, 0, h->stream>>>(
          nu, np, h->q, F.ns, F.R, C.ns, C.R, F.Pu_p, F.Pu_c, F.Pu_v, F.Pp_p, F.Pp_c, F.Pp_v, dc, df, 1, nb, C.N, F.N);
  }
}

template <typename T>
void coarse(stfem_h h, const T *b, T *x, int nb = 1) {
  const long n = levels<T>(h)[0].N;
  Launch G_(h, STFEM_KCLASS_COARSE, (double)n * n * 8.0 + 2.0 * n * sizeof(T) * nb, 2.0 * n * n * nb);
  k_coarse<T><<<grid_for(n * 32, 256) * nb, 256, 0, h->stream>>>(n, h->coarse_inv, b, x, nb);
}

// V-cycle on level l for A_l d_l = b_l (both in the level's buffers), d from
// 0; nb columns (column stride N of each level) at once.
template <typename T>
void vcycle(stfem_h h, int l, int nb = 1) {
  std::vector<DLevel<T>> &Ls = levels<T>(h);
  if (l == 0) {
    coarse<T>(h, Ls[0].b, Ls[0].d, nb);
    return;
  }
  DLevel<T> &L = Ls[l];
  const TimeCoef<T> tc = time_coef<T>(h->T, h->tau);
  smooth<T>(h, l, h->nsweeps, true, nb);
  launch_spmv<T>(h, L, tc, L.d, L.b, L.r, 1, nb);
  restrict_to<T>(h, l, L.r, Ls[l - 1].b, nb);
  vcycle<T>(h, l - 1, nb);
  prolongate_add<T>(h, l, Ls[l - 1].d, L.d, nb);
  smooth<T>(h, l, h->nsweeps, false, nb);
}

// z = M^{-1} v with one V-cycle in the GMG precision; v, z FP64 (z may be FP32 storage)
int precondition(stfem_h h, const double *v, double *zd, float *zf) {
  const int L = h->nlev - 1;
  cudaStream_t s = h->stream;
  if (h->precision == STFEM_FP64) {
    DLevel<double> &F = h->L64[L];
    CK(cudaMemcpyAsync(F.b, v, F.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    vcycle<double>(h, L);
    CK(cudaMemcpyAsync(zd, F.d, F.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    DLevel<float> &F = h->L32[L];
    {
      Launch G_(h, STFEM_KCLASS_OTHER, F.N * 12.0, 0.0);
      k_convert<double, float><<<grid_for(F.N, 256), 256, 0, s>>>(F.N, v, F.b);
    }
    vcycle<float>(h, L);
    if (zf) CK(cudaMemcpyAsync(zf, F.d, F.N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (zd) {
      Launch G_(h, STFEM_KCLASS_OTHER, F.N * 12.0, 0.0);
      k_convert<float, double><<<grid_for(F.N, 256), 256, 0, s>>>(F.N, F.d, zd);
    }
  }
  CK(cudaGetLastError());
  return 0;
}

// dots out[0..k) = V_v . w on device (deterministic two-stage reduction)
void multidot(stfem_h h, int k, const double *V, long ldV, const double *w, long n, double *out) {
  const int nbk = h->dot_blocks;
  dim3 grid(nbk, (k + DOT_NV - 1) / DOT_NV);
  {
    Launch G_(h, STFEM_KCLASS_BLAS1, (double)(k + 1) * n * 8.0, 2.0 * k * n);
    k_multidot<<<grid, DOT_THREADS, 0, h->stream>>>(k, V, ldV, w, n, h->partial);
  }
  {
    Launch G_(h, STFEM_KCLASS_OTHER, (double)k * nbk * 8.0, (double)k * nbk);
    k_reduce_partials<<<k, 256, 0, h->stream>>>(nbk, h->partial, out);
  }
}

// w <- w - V h (k vectors), then out = V^T w (mode 0, k values) or
// out = w . w (mode 1): one pass over V and w, fixed-order reduction.
void axpy_dot(stfem_h h, int k, const double *V, long ldV, const double *hvec, double *w, long n, double *out,
              int mode) {
  const int nbk = h->dot_blocks;
  {
    Launch G_(h, STFEM_KCLASS_BLAS1, (double)(k + 2) * n * 8.0, 2.0 * k * n * (mode == 0 ? 2 : 1) + 2.0 * n);
    // the register blocks run KB >= k multiply-adds per entry: KB in steps of 4
#define STFEM_AXPY_DOT(KB)                                                                                \
  k_axpy_dot<KB><<<nbk, DOT_THREADS, 0, h->stream>>>(k, V, ldV, hvec, w, n, h->partial, mode)
    if (k <= 4) STFEM_AXPY_DOT(4);
    else if (k <= 8) STFEM_AXPY_DOT(8);
    else if (k <= 12) STFEM_AXPY_DOT(12);
    else if (k <= 16) STFEM_AXPY_DOT(16);
    else if (k <= 20) STFEM_AXPY_DOT(20);
    else if (k <= 24) STFEM_AXPY_DOT(24);
    else if (k <= 28) STFEM_AXPY_DOT(28);
    else STFEM_AXPY_DOT(32);
#undef STFEM_AXPY_DOT
  }
  {
    const int nout = mode == 0 ? k : 1;
    Launch G_(h, STFEM_KCLASS_OTHER, (double)nout * nbk * 8.0, (double)nout * nbk);
    k_reduce_partials<<<nout, 256, 0, h->stream>>>(nbk, h->partial, out);
  }
}

int read_scalar(stfem_h h, const double *dev, double *host) {
  CK(cudaMemcpyAsync(h->status_host, dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *host = h->status_host[0];
  return 0;
}

int ensure_workspace(stfem_h h, int m) {
  if (m <= h->mcap) return 0;
  if (m > MAXM) {
    h->err = "restart length above the supported maximum";
    return STFEM_ERR_ARG;
  }
  const long N = h->L64.back().N;
  CKR(dalloc(h, &h->V, (size_t)(m + 1) * N));
  if (h->precision == STFEM_MIXED) {
    CKR(dalloc(h, &h->Zf, (size_t)m * N));
  } else {
    CKR(dalloc(h, &h->Zd, (size_t)m * N));
  }
  CKR(dalloc(h, &h->H, (size_t)(m + 1) * m));
  CKR(dalloc(h, &h->cs, m));
  CKR(dalloc(h, &h->sn, m));
  CKR(dalloc(h, &h->g, m + 1));
  CKR(dalloc(h, &h->y, m));
  CKR(dalloc(h, &h->h1, m + 1));
  CKR(dalloc(h, &h->h2, m + 1));
  h->mcap = m;
  for (auto &g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.assign(m, stfem_ctx::GraphRec());
  return 0;
}

// The two halves of FGMRES iteration j around its V-cycle.  iter_pre: the
// V-cycle input v_j in the GMG precision.  iter_post: z_j = the V-cycle
// output kept for the solution update, w = A z_j, classical Gram-Schmidt
// twice (h1 = V^T w; w -= V h1 and h2 = V^T w in one pass; w -= V h2 and
// ||w||^2 in one pass), the Givens update, a copy of the status
// {|g_{j+1}|, h_{j+1,j}} to pinned host memory, and v_{j+1} = w / h_{j+1,j}
// (unused when the host stops at j).
int iter_pre(stfem_h h, int j) {
  const int L = h->nlev - 1;
  const long N = h->L64.back().N;
  const double *vj = h->V + (long)j * N;
  cudaStream_t s = h->stream;
  if (h->precision == STFEM_FP64) {
    CK(cudaMemcpyAsync(h->L64[L].b, vj, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    Launch G_(h, STFEM_KCLASS_OTHER, N * 12.0, 0.0);
    k_convert<double, float><<<grid_for(N, 256), 256, 0, s>>>(N, vj, h->L32[L].b);
  }
  return 0;
}

int iter_post(stfem_h h, int j, int m1) {
  DLevel<double> &F = h->L64.back();
  const long N = F.N;
  const int L = h->nlev - 1;
  const TimeCoef<double> tc = time_coef<double>(h->T, h->tau);
  cudaStream_t s = h->stream;
  const int nb = grid_for(N, 256);
  double *w = h->w;
  if (h->precision == STFEM_FP64) {
    double *zj = h->Zd + (long)j * N;
    CK(cudaMemcpyAsync(zj, h->L64[L].d, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    launch_spmv<double>(h, F, tc, zj, nullptr, w, 0);
  } else {
    float *zf = h->Zf + (long)j * N;
    CK(cudaMemcpyAsync(zf, h->L32[L].d, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (F.has_df) {
      // z_j is the FP32 V-cycle output: exact in FP32, so A z_j in double-float
      launch_spmv_df(h, F, tc, zf, w);
    } else {
      {
        Launch G_(h, STFEM_KCLASS_OTHER, N * 12.0, 0.0);
        k_convert<float, double><<<grid_for(N, 256), 256, 0, s>>>(N, h->L32[L].d, h->zt);
      }
      launch_spmv<double>(h, F, tc, h->zt, nullptr, w, 0);
    }
  }
  multidot(h, j + 1, h->V, N, w, N, h->h1);
  axpy_dot(h, j + 1, h->V, N, h->h1, w, N, h->h2, 0);
  axpy_dot(h, j + 1, h->V, N, h->h2, w, N, h->hn2, 1);
  {
    Launch G_(h, STFEM_KCLASS_OTHER, (double)(4 * j + 8) * 8.0, (double)(6 * j + 10));
    k_givens<<<1, 1, 0, s>>>(j, m1, h->h1, h->h2, h->hn2, h->H, h->cs, h->sn, h->g, h->hnorm, h->status);
  }
  CK(cudaMemcpyAsync(h->status_host, h->status, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (j + 1 < m1) {
    Launch G_(h, STFEM_KCLASS_BLAS1, N * 16.0, (double)N);
    k_div<<<nb, 256, 0, s>>>(N, w, h->V + (long)(j + 1) * N, h->hnorm, 0.0);
  }
  CK(cudaGetLastError());
  return 0;
}

// All work of FGMRES iteration j (Sec. 4): z_j = M^{-1} v_j (one V-cycle) and
// the rest of iter_post.  Only stream-ordered work: it can be captured into a
// graph.
int enqueue_iteration(stfem_h h, int j, int m1) {
  CKR(iter_pre(h, j));
  if (h->precision == STFEM_FP64)
    vcycle<double>(h, h->nlev - 1);
  else
    vcycle<float>(h, h->nlev - 1);
  return iter_post(h, j, m1);
}

// Runs the work enqueue() issues from its captured graph gv[j] (captured on
// first use), or eagerly when profiling (per-launch events) or on the legacy
// stream.
template <typename F>
int run_captured(stfem_h h, std::vector<stfem_ctx::GraphRec> &gv, int j, F enqueue) {
  const bool graphs = h->use_graphs && !h->prof && h->stream != 0 && j < (int)gv.size();
  if (!graphs) return enqueue();
  stfem_ctx::GraphRec &g = gv[j];
  if (!g.exec) {
    stfem_ctx::KStat before[STFEM_KCLASS_COUNT];
    for (int k = 0; k < STFEM_KCLASS_COUNT; ++k) before[k] = h->kstat[k];
    const long long l0 = h->launches;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->use_graphs = false;
      return enqueue();
    }
    const int rc = enqueue();
    const cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
    if (rc < 0) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess || cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      g.exec = nullptr;
      h->use_graphs = false;
      for (int k = 0; k < STFEM_KCLASS_COUNT; ++k) h->kstat[k] = before[k];
      h->launches = l0;
      return enqueue();
    }
    cudaGraphDestroy(graph);
    // the capture only recorded the launches: keep their accounting with the
    // graph and count them when it runs
    for (int k = 0; k < STFEM_KCLASS_COUNT; ++k) {
      g.delta[k].launches = h->kstat[k].launches - before[k].launches;
      g.delta[k].bytes = h->kstat[k].bytes - before[k].bytes;
      g.delta[k].flops = h->kstat[k].flops - before[k].flops;
      h->kstat[k] = before[k];
    }
    g.launches = h->launches - l0;
    h->launches = l0;
  }
  CK(cudaGraphLaunch(g.exec, h->stream));
  for (int k = 0; k < STFEM_KCLASS_COUNT; ++k) {
    h->kstat[k].launches += g.delta[k].launches;
    h->kstat[k].bytes += g.delta[k].bytes;
    h->kstat[k].flops += g.delta[k].flops;
  }
  h->launches += g.launches;
  return 0;
}

int run_iteration(stfem_h h, int j, int m1) {
  return run_captured(h, h->graphs, j, [&]() { return enqueue_iteration(h, j, m1); });
}

int fgmres(stfem_h h, const double *b, double *x, double tol, int m, int max_it, int *iters, double *relres,
           double *absres) {
  CKR(ensure_workspace(h, m));
  DLevel<double> &F = h->L64.back();
  const long N = F.N;
  const TimeCoef<double> tc = time_coef<double>(h->T, h->tau);
  cudaStream_t s = h->stream;
  const int nb = grid_for(N, 256);
  h->hist.clear();
  *iters = 0;
  *relres = 0.0;
  *absres = 0.0;
  launch_spmv<double>(h, F, tc, x, b, h->rvec, 1);
  multidot(h, 1, h->rvec, N, h->rvec, N, h->hn2);
  double beta0sq;
  CKR(read_scalar(h, h->hn2, &beta0sq));
  const double beta0 = std::sqrt(beta0sq);
  *absres = beta0;
  h->hist.push_back(1.0);
  if (!std::isfinite(beta0)) {
    h->err = "initial residual is not finite";
    return STFEM_ERR_BREAKDOWN;
  }
  const double bound = h->stop == STFEM_STOP_ABSOLUTE ? tol : tol * beta0;
  if (beta0 == 0.0 || beta0 <= bound) {
    *relres = beta0 > 0.0 ? 1.0 : 0.0;
    return STFEM_OK;
  }
  double beta = beta0;
  int it = 0;
  const int m1 = m + 1;
  for (;;) {
    {
      Launch G_(h, STFEM_KCLASS_BLAS1, N * 16.0, (double)N);
      k_div<<<nb, 256, 0, s>>>(N, h->rvec, h->V, nullptr, beta);
    }
    {
      Launch G_(h, STFEM_KCLASS_OTHER, 8.0, 0.0);
      k_set<<<1, 1, 0, s>>>(h->g, beta);
    }
    int jlast = -1;
    bool stop = false;
    for (int j = 0; j < m; ++j) {
      CKR(run_iteration(h, j, m1));
      CK(cudaStreamSynchronize(s));
      CK(cudaGetLastError());
      const double res = h->status_host[0], hn = h->status_host[1];
      if (!std::isfinite(res) || !std::isfinite(hn)) {
        h->err = "FGMRES breakdown: non-finite Hessenberg entry";
        *iters = it;
        return STFEM_ERR_BREAKDOWN;
      }
      ++it;
      jlast = j;
      h->hist.push_back(res / beta0);
      if (res <= bound || it >= max_it || hn == 0.0) {
        stop = true;
        break;
      }
    }
    const int kk = jlast + 1;
    {
      Launch G_(h, STFEM_KCLASS_OTHER, (double)kk * kk * 8.0, (double)kk * kk);
      k_backsolve<<<1, 1, 0, s>>>(kk, m1, h->H, h->g, h->y);
    }
    {
      Launch G_(h, STFEM_KCLASS_BLAS1, (double)N * (16.0 + kk * (h->precision == STFEM_FP64 ? 8.0 : 4.0)),
                2.0 * kk * N);
      if (h->precision == STFEM_FP64)
        k_update_x<double><<<nb, 256, 0, s>>>(N, kk, h->Zd, N, h->y, x);
      else
        k_update_x<float><<<nb, 256, 0, s>>>(N, kk, h->Zf, N, h->y, x);
    }
    launch_spmv<double>(h, F, tc, x, b, h->rvec, 1);
    multidot(h, 1, h->rvec, N, h->rvec, N, h->hn2);
    double rr;
    CKR(read_scalar(h, h->hn2, &rr));
    const double res = std::sqrt(rr);
    *iters = it;
    *relres = res / beta0;
    *absres = res;
    if (!std::isfinite(res)) {
      h->err = "FGMRES breakdown: non-finite residual";
      return STFEM_ERR_BREAKDOWN;
    }
    if (res <= bound) return STFEM_OK;
    if (it >= max_it) return STFEM_NOT_CONVERGED;
    (void)stop;
    beta = res;
  }
}

// ---------------------------------------------------------------- several right-hand sides
// Columns c = 0..nb-1 of the batch: one flexible GMRES per column (its own
// Krylov basis, Hessenberg matrix and rotations), all columns advanced in
// lockstep so that the V-cycle preconditions the nb vectors v_j together
// (the patch inverses and level operators are read once per sweep for all
// columns).  A column that has met its bound keeps iterating harmlessly until
// the others finish the cycle; it uses only its first k_c iterations.
struct BatchCol {
  double *V, *H, *cs, *sn, *g, *y, *h1, *h2, *hnorm, *hn2, *status;
};

BatchCol batch_col(stfem_h h, int c) {
  stfem_ctx::Batch &B = h->bt;
  const long N = h->L64.back().N;
  const int m = B.m, m1 = m + 1;
  double *sm = B.small + (long)c * B.sw;
  BatchCol k;
  k.V = B.V + (long)c * m1 * N;
  k.H = sm;
  k.cs = k.H + (long)m1 * m;
  k.sn = k.cs + m;
  k.g = k.sn + m;
  k.y = k.g + m1;
  k.h1 = k.y + m;
  k.h2 = k.h1 + m1;
  k.hnorm = k.h2 + m1;
  k.hn2 = B.norms + c;
  k.status = B.norms + h->nrhs_cap + 2 * c;
  return k;
}

int ensure_batch_workspace(stfem_h h, int m) {
  stfem_ctx::Batch &B = h->bt;
  if (m > MAXM) {
    h->err = "restart length above the supported maximum";
    return STFEM_ERR_ARG;
  }
  if (m <= B.m) return 0;
  const long N = h->L64.back().N;
  const int nb = h->nrhs_cap, m1 = m + 1;
  CKR(dalloc(h, &B.V, (size_t)nb * m1 * N));
  if (h->precision == STFEM_MIXED) {
    CKR(dalloc(h, &B.Zf, (size_t)nb * m * N));
  } else {
    CKR(dalloc(h, &B.Zd, (size_t)nb * m * N));
  }
  CKR(dalloc(h, &B.zt, (size_t)nb * N));
  CKR(dalloc(h, &B.w, (size_t)nb * N));
  CKR(dalloc(h, &B.rvec, (size_t)nb * N));
  if (!B.rhs) {
    CKR(dalloc(h, &B.rhs, (size_t)nb * N));
    CKR(dalloc(h, &B.xs, (size_t)nb * N));
  }
  B.sw = (long)m1 * m + 2L * m + m1 + m + 2L * m1 + 1;
  CKR(dalloc(h, &B.small, (size_t)nb * B.sw));
  if (!B.norms) {
    CKR(dalloc(h, &B.norms, (size_t)3 * nb));
    CK(cudaHostAlloc((void **)&B.host, (size_t)3 * nb * sizeof(double), cudaHostAllocDefault));
  }
  B.m = m;
  for (auto &g : B.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  B.graphs.assign(m, stfem_ctx::GraphRec());
  B.nb = 0;
  return 0;
}

// Same as enqueue_iteration, for nb columns: one batched V-cycle and one
// batched SpMV, then CGS2 and the Givens update per column; the statuses of
// all columns are copied to pinned memory at once.
int enqueue_iteration_batch(stfem_h h, int j, int m1, int nb) {
  stfem_ctx::Batch &B = h->bt;
  DLevel<double> &F = h->L64.back();
  const long N = F.N;
  const int m = m1 - 1;
  const TimeCoef<double> tc = time_coef<double>(h->T, h->tau);
  cudaStream_t s = h->stream;
  const int nbk = grid_for(N, 256);
  const int L = h->nlev - 1;
  const double *vj = B.V + (long)j * N; // column stride m1 * N
  const double *zsp = nullptr;          // z_j of all columns, column stride N, FP64
  if (h->precision == STFEM_FP64) {
    DLevel<double> &G = h->L64[L];
    {
      Launch G_(h, STFEM_KCLASS_OTHER, N * 16.0 * nb, 0.0);
      k_copy_cols<double, double><<<nbk * nb, 256, 0, s>>>(N, nb, vj, (long)m1 * N, G.b, N);
    }
    vcycle<double>(h, L, nb);
    {
      Launch G_(h, STFEM_KCLASS_OTHER, N * 16.0 * nb, 0.0);
      k_copy_cols<double, double><<<nbk * nb, 256, 0, s>>>(N, nb, G.d, N, B.Zd + (long)j * N, (long)m * N);
    }
    zsp = G.d;
  } else {
    DLevel<float> &G = h->L32[L];
    {
      Launch G_(h, STFEM_KCLASS_OTHER, N * 12.0 * nb, 0.0);
      k_copy_cols<double, float><<<nbk * nb, 256, 0, s>>>(N, nb, vj, (long)m1 * N, G.b, N);
    }
    vcycle<float>(h, L, nb);
    {
      Launch G_(h, STFEM_KCLASS_OTHER, N * 8.0 * nb, 0.0);
      k_copy_cols<float, float><<<nbk * nb, 256, 0, s>>>(N, nb, G.d, N, B.Zf + (long)j * N, (long)m * N);
    }
    if (F.has_df) {
      launch_spmv_df(h, F, tc, G.d, B.w, nb);
    } else {
      {
        Launch G_(h, STFEM_KCLASS_OTHER, N * 12.0 * nb, 0.0);
        k_copy_cols<float, double><<<nbk * nb, 256, 0, s>>>(N, nb, G.d, N, B.zt, N);
      }
      zsp = B.zt;
    }
  }
  if (zsp) launch_spmv<double>(h, F, tc, zsp, nullptr, B.w, 0, nb);
  for (int c = 0; c < nb; ++c) {
    const BatchCol k = batch_col(h, c);
    double *w = B.w + (long)c * N;
    multidot(h, j + 1, k.V, N, w, N, k.h1);
    axpy_dot(h, j + 1, k.V, N, k.h1, w, N, k.h2, 0);
    axpy_dot(h, j + 1, k.V, N, k.h2, w, N, k.hn2, 1);
    {
      Launch G_(h, STFEM_KCLASS_OTHER, (double)(4 * j + 8) * 8.0, (double)(6 * j + 10));
      k_givens<<<1, 1, 0, s>>>(j, m1, k.h1, k.h2, k.hn2, k.H, k.cs, k.sn, k.g, k.hnorm, k.status);
    }
  }
  CK(cudaMemcpyAsync(B.host + h->nrhs_cap, B.norms + h->nrhs_cap, 2 * (size_t)nb * sizeof(double),
                     cudaMemcpyDeviceToHost, s));
  if (j + 1 < m1)
    for (int c = 0; c < nb; ++c) {
      const BatchCol k = batch_col(h, c);
      Launch G_(h, STFEM_KCLASS_BLAS1, N * 16.0, (double)N);
      k_div<<<nbk, 256, 0, s>>>(N, B.w + (long)c * N, k.V + (long)(j + 1) * N, k.hnorm, 0.0);
    }
  return 0;
}

// r = b - A x for nb columns and ||r_c||^2 -> host[c]
int batch_residuals(stfem_h h, int nb, const double *b, const double *x) {
  stfem_ctx::Batch &B = h->bt;
  DLevel<double> &F = h->L64.back();
  const long N = F.N;
  const TimeCoef<double> tc = time_coef<double>(h->T, h->tau);
  launch_spmv<double>(h, F, tc, x, b, B.rvec, 1, nb);
  for (int c = 0; c < nb; ++c) multidot(h, 1, B.rvec + (long)c * N, N, B.rvec + (long)c * N, N, B.norms + c);
  CK(cudaMemcpyAsync(B.host, B.norms, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return 0;
}

// Flexible GMRES(m) for nb right-hand sides (device, column stride N):
// every column is solved as by fgmres() alone (same stopping rule per
// column); iters[c], relres[c] per column.  Returns the worst status.
int fgmres_batch(stfem_h h, int nb, const double *b, double *x, double tol, int m, int max_it, int *iters,
                 double *relres) {
  CKR(ensure_batch_workspace(h, m));
  stfem_ctx::Batch &B = h->bt;
  if (B.nb != nb) { // graphs hold the column count in their launches
    for (auto &g : B.graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    B.graphs.assign(B.m, stfem_ctx::GraphRec());
    B.nb = nb;
  }
  DLevel<double> &F = h->L64.back();
  const long N = F.N;
  cudaStream_t s = h->stream;
  const int nbk = grid_for(N, 256);
  const int m1 = m + 1;
  std::vector<double> beta0(nb), bound(nb), beta(nb);
  std::vector<int> active(nb, 0), it(nb, 0), kk(nb, 0), done(nb, 0);
  CKR(batch_residuals(h, nb, b, x));
  int worst = STFEM_OK;
  for (int c = 0; c < nb; ++c) {
    beta0[c] = std::sqrt(B.host[c]);
    if (!std::isfinite(beta0[c])) {
      h->err = "initial residual is not finite";
      return STFEM_ERR_BREAKDOWN;
    }
    bound[c] = h->stop == STFEM_STOP_ABSOLUTE ? tol : tol * beta0[c];
    active[c] = beta0[c] > 0.0 && beta0[c] > bound[c];
    beta[c] = beta0[c];
    iters[c] = 0;
    relres[c] = beta0[c] > 0.0 && !active[c] ? 1.0 : 0.0;
  }
  for (;;) {
    int nact = 0;
    for (int c = 0; c < nb; ++c) nact += active[c];
    if (nact == 0) break;
    for (int c = 0; c < nb; ++c) {
      const BatchCol k = batch_col(h, c);
      const double bc = active[c] ? beta[c] : 0.0; // finished columns run on zeros
      {
        Launch G_(h, STFEM_KCLASS_BLAS1, N * 16.0, (double)N);
        k_div<<<nbk, 256, 0, s>>>(N, B.rvec + (long)c * N, k.V, nullptr, bc);
      }
      {
        Launch G_(h, STFEM_KCLASS_OTHER, 8.0, 0.0);
        k_set<<<1, 1, 0, s>>>(k.g, bc);
      }
      done[c] = !active[c];
      kk[c] = 0;
    }
    for (int j = 0; j < m; ++j) {
      CKR(run_captured(h, B.graphs, j, [&]() { return enqueue_iteration_batch(h, j, m1, nb); }));
      CK(cudaStreamSynchronize(s));
      CK(cudaGetLastError());
      bool all = true;
      for (int c = 0; c < nb; ++c) {
        if (done[c]) continue;
        const double res = B.host[h->nrhs_cap + 2 * c], hn = B.host[h->nrhs_cap + 2 * c + 1];
        if (!std::isfinite(res) || !std::isfinite(hn)) {
          h->err = "FGMRES breakdown: non-finite Hessenberg entry in column " + std::to_string(c);
          return STFEM_ERR_BREAKDOWN;
        }
        ++it[c];
        kk[c] = j + 1;
        if (res <= bound[c] || it[c] >= max_it || hn == 0.0) done[c] = 1;
        all = all && done[c];
      }
      if (all) break;
    }
    for (int c = 0; c < nb; ++c) {
      if (!active[c] || kk[c] == 0) continue;
      const BatchCol k = batch_col(h, c);
      {
        Launch G_(h, STFEM_KCLASS_OTHER, (double)kk[c] * kk[c] * 8.0, (double)kk[c] * kk[c]);
        k_backsolve<<<1, 1, 0, s>>>(kk[c], m1, k.H, k.g, k.y);
      }
      Launch G_(h, STFEM_KCLASS_BLAS1, (double)N * (16.0 + kk[c] * (h->precision == STFEM_FP64 ? 8.0 : 4.0)),
                2.0 * kk[c] * N);
      if (h->precision == STFEM_FP64)
        k_update_x<double><<<nbk, 256, 0, s>>>(N, kk[c], B.Zd + (long)c * m * N, N, k.y, x + (long)c * N);
      else
        k_update_x<float><<<nbk, 256, 0, s>>>(N, kk[c], B.Zf + (long)c * m * N, N, k.y, x + (long)c * N);
    }
    CKR(batch_residuals(h, nb, b, x));
    for (int c = 0; c < nb; ++c) {
      if (!active[c]) continue;
      const double res = std::sqrt(B.host[c]);
      if (!std::isfinite(res)) {
        h->err = "FGMRES breakdown: non-finite residual in column " + std::to_string(c);
        return STFEM_ERR_BREAKDOWN;
      }
      iters[c] = it[c];
      relres[c] = res / beta0[c];
      beta[c] = res;
      if (res <= bound[c]) {
        active[c] = 0;
      } else if (it[c] >= max_it) {
        active[c] = 0;
        worst = STFEM_NOT_CONVERGED;
      }
    }
  }
  return worst;
}

// A bounded wait inside a kernel timed out (reported through h->dev_err):
// the flag is cleared again, so that the handle's next call starts clean.
int check_dev_err(stfem_h h) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (e) {
    CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const char *who = e == 1 ? "streaming patch apply, producer" : e == 2 ? "streaming patch apply, consumer"
                                                                         : "tensor-core patch apply";
    h->err = std::string("a bounded wait timed out (") + who + ", code " + std::to_string(e) + ")";
    return STFEM_ERR_TIMEOUT;
  }
  return 0;
}

// Drops the captured per-iteration graphs (their kernels hold launch
// parameters that a setting of the handle has changed); they are captured
// again on their next use.
void drop_graphs(stfem_h h) {
  for (auto &g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.assign(h->graphs.size(), stfem_ctx::GraphRec());
  for (auto &g : h->bt.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->bt.graphs.assign(h->bt.graphs.size(), stfem_ctx::GraphRec());
}

int check_level(stfem_h h, int level, bool allow_fine_alias) {
  if (level == -1 && allow_fine_alias) return 0;
  if (level < 0 || level >= h->nlev) {
    h->err = "level out of range";
    return STFEM_ERR_ARG;
  }
  return 0;
}

int require_gmg(stfem_h h) {
  if (h->precision < 0) {
    h->err = "stfem_gmg_setup has not been called";
    return STFEM_ERR_STATE;
  }
  return 0;
}

// copy an FP64 ABI vector into a level buffer of type T (and back)
template <typename T>
void to_level(stfem_h h, const double *src, T *dst, long n) {
  Launch G_(h, STFEM_KCLASS_OTHER, n * (8.0 + sizeof(T)), 0.0);
  k_convert<double, T><<<grid_for(n, 256), 256, 0, h->stream>>>(n, src, dst);
}
template <typename T>
void from_level(stfem_h h, const T *src, double *dst, long n) {
  Launch G_(h, STFEM_KCLASS_OTHER, n * (8.0 + sizeof(T)), 0.0);
  k_convert<T, double><<<grid_for(n, 256), 256, 0, h->stream>>>(n, src, dst);
}

template <typename T>
int apply_t(stfem_h h, int level, const double *x, double *y) {
  DLevel<T> &L = levels<T>(h)[level];
  const TimeCoef<T> tc = time_coef<T>(h->T, h->tau);
  to_level<T>(h, x, L.d, L.N);
  launch_spmv<T>(h, L, tc, L.d, nullptr, L.r, 0);
  from_level<T>(h, L.r, y, L.N);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

// nb columns of b and d (column stride N of the level)
template <typename T>
int smooth_t(stfem_h h, int level, const double *b, double *d, int nsw, int zero_init, int nb = 1) {
  DLevel<T> &L = levels<T>(h)[level];
  if (nb == 1) {
    to_level<T>(h, b, L.b, L.N);
    if (!zero_init) to_level<T>(h, d, L.d, L.N);
  } else {
    Launch G_(h, STFEM_KCLASS_OTHER, L.N * (8.0 + sizeof(T)) * nb * (zero_init ? 1 : 2), 0.0);
    k_copy_cols<double, T><<<grid_for(L.N, 256) * nb, 256, 0, h->stream>>>(L.N, nb, b, L.N, L.b, L.N);
    if (!zero_init) k_copy_cols<double, T><<<grid_for(L.N, 256) * nb, 256, 0, h->stream>>>(L.N, nb, d, L.N, L.d, L.N);
  }
  smooth<T>(h, level, nsw, zero_init != 0, nb);
  if (nb == 1) {
    from_level<T>(h, L.d, d, L.N);
  } else {
    Launch G_(h, STFEM_KCLASS_OTHER, L.N * (8.0 + sizeof(T)) * nb, 0.0);
    k_copy_cols<T, double><<<grid_for(L.N, 256) * nb, 256, 0, h->stream>>>(L.N, nb, L.d, L.N, d, L.N);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  CKR(check_dev_err(h));
  return 0;
}

template <typename T>
int transfer_t(stfem_h h, int level, const double *in, double *out, bool restrict_dir) {
  std::vector<DLevel<T>> &Ls = levels<T>(h);
  DLevel<T> &F = Ls[level], &C = Ls[level - 1];
  if (restrict_dir) {
    to_level<T>(h, in, F.r, F.N);
    restrict_to<T>(h, level, F.r, C.b);
    from_level<T>(h, C.b, out, C.N);
  } else {
    to_level<T>(h, in, C.d, C.N);
    to_level<T>(h, out, F.d, F.N);
    prolongate_add<T>(h, level, C.d, F.d);
    from_level<T>(h, F.d, out, F.N);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

int build_load_tables(stfem_h h) {
  const stfem::Level &L = h->hl.back();
  const stfem::Box &b = L.box;
  const int d = b.dim, nq1 = h->r + 2;
  stfem::Rule g = stfem::gauss01(nq1);
  std::vector<double> qx, qw, fx, fw;
  int nz = d > 2 ? nq1 : 1, ny = d > 1 ? nq1 : 1;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nq1; ++x) {
        qx.push_back(g.x[x]);
        qx.push_back(d > 1 ? g.x[y] : 0.0);
        qx.push_back(d > 2 ? g.x[z] : 0.0);
        qw.push_back(g.w[x] * (d > 1 ? g.w[y] : 1.0) * (d > 2 ? g.w[z] : 1.0) * b.vol);
      }
  if (d == 3) {
    const double area = b.h[0] * b.h[1];
    for (int y = 0; y < nq1; ++y)
      for (int x = 0; x < nq1; ++x) {
        fx.push_back(g.x[x]);
        fx.push_back(g.x[y]);
        fx.push_back(1.0);
        fw.push_back(g.w[x] * g.w[y] * area);
      }
  }
  auto tab = [&](const stfem::Lattice &lat, const std::vector<double> &pts) {
    const int m1 = lat.m + 1;
    int nl = 1;
    for (int i = 0; i < d; ++i) nl *= m1;
    const int np = (int)pts.size() / 3;
    std::vector<double> out((size_t)np * nl);
    std::vector<double> v(m1), dv(m1);
    for (int qq = 0; qq < np; ++qq) {
      double vals[3][16];
      for (int i = 0; i < d; ++i) {
        stfem::lagrange(lat.ref, pts[qq * 3 + i], v.data(), dv.data());
        for (int j = 0; j < m1; ++j) vals[i][j] = v[j];
      }
      for (int l = 0; l < nl; ++l) {
        int t = l;
        double p = 1.0;
        for (int i = 0; i < d; ++i) {
          p *= vals[i][t % m1];
          t /= m1;
        }
        out[(size_t)qq * nl + l] = p;
      }
    }
    return out;
  };
  std::vector<double> phiU = tab(L.U, qx), phiP;
  std::vector<double> fphiU = d == 3 ? tab(L.U, fx) : std::vector<double>(1, 0.0);
  int nlu = 1, nlp = 1;
  for (int i = 0; i < d; ++i) {
    nlu *= h->r + 1;
    nlp *= h->r;
  }
  LoadTables &lt = h->lt;
  std::vector<double> pqx, pqw, phiPP;
  if (L.pdisc) {
    nlp = stfem::disc_basis(h->r - 1, d, qx.data(), (int)qw.size(), &phiP);
    // projection rule: Gauss with r + 3 points per direction (weights of the
    // reference cell: the cell measure cancels in the projection)
    const int np1 = h->r + 3;
    stfem::Rule gp = stfem::gauss01(np1);
    const int pz = d > 2 ? np1 : 1, py = d > 1 ? np1 : 1;
    for (int z = 0; z < pz; ++z)
      for (int y = 0; y < py; ++y)
        for (int x = 0; x < np1; ++x) {
          pqx.push_back(gp.x[x]);
          pqx.push_back(d > 1 ? gp.x[y] : 0.0);
          pqx.push_back(d > 2 ? gp.x[z] : 0.0);
          pqw.push_back(gp.w[x] * (d > 1 ? gp.w[y] : 1.0) * (d > 2 ? gp.w[z] : 1.0));
        }
    stfem::disc_basis(h->r - 1, d, pqx.data(), (int)pqw.size(), &phiPP);
  } else {
    phiP = tab(L.P, qx);
    pqx.assign(3, 0.0);
    pqw.assign(1, 0.0);
    phiPP.assign(1, 0.0);
  }
  lt.pdisc = L.pdisc ? 1 : 0;
  lt.npq = L.pdisc ? (int)pqw.size() : 0;
  lt.nq = (int)qw.size();
  lt.nlu = nlu;
  lt.nlp = nlp;
  lt.nqf = (int)fw.size();
  double *p;
  CKR(upload(h, &p, qx)); lt.qx = p;
  CKR(upload(h, &p, qw)); lt.qw = p;
  CKR(upload(h, &p, phiU)); lt.phiU = p;
  CKR(upload(h, &p, phiP)); lt.phiP = p;
  CKR(upload(h, &p, fx.empty() ? std::vector<double>(3, 0.0) : fx)); lt.fx = p;
  CKR(upload(h, &p, fw.empty() ? std::vector<double>(1, 0.0) : fw)); lt.fw = p;
  CKR(upload(h, &p, fphiU)); lt.fphiU = p;
  CKR(upload(h, &p, L.coef.lam)); lt.lam = p;
  CKR(upload(h, &p, L.coef.mu)); lt.mu = p;
  {
    std::vector<double> Kt((size_t)L.box.ncell * 9, 0.0);
    for (long c = 0; c < L.box.ncell; ++c)
      for (int a = 0; a < d; ++a)
        for (int b2 = 0; b2 < d; ++b2)
          Kt[(size_t)c * 9 + a * 3 + b2] = L.coef.K.empty() ? (a == b2 ? L.coef.kap[c] : 0.0)
                                                            : L.coef.K[((size_t)c * d + a) * d + b2];
    CKR(upload(h, &p, Kt));
    lt.Kt = p;
  }
  CKR(upload(h, &p, pqx)); lt.pqx = p;
  CKR(upload(h, &p, pqw)); lt.pqw = p;
  CKR(upload(h, &p, phiPP)); lt.phiPP = p;
  // face rule and basis data of the boundary data terms
  stfem::FaceTables ft;
  stfem::face_tables(L, &ft);
  if (ft.nu != nlu || ft.np != nlp) {
    h->err = "face tables do not match the load tables";
    return STFEM_ERR_STATE;
  }
  lt.nqd = ft.npts;
  CKR(upload(h, &p, ft.x)); lt.dfx = p;
  CKR(upload(h, &p, ft.w)); lt.dfw = p;
  CKR(upload(h, &p, ft.U)); lt.dfU = p;
  CKR(upload(h, &p, ft.dU)); lt.dfdU = p;
  CKR(upload(h, &p, ft.P)); lt.dfP = p;
  CKR(upload(h, &p, ft.dP)); lt.dfdP = p;
  return 0;
}

int fail_setup(stfem_h h, int rc) {
  g_setup_err = h->err;
  stfem_destroy(h);
  return rc;
}

} // namespace

int stfem::block_apply_level(const stfem::Level &L, int q, const double *Dt, const double *W, const double *x,
                             double *y, std::string *err) {
  NodeBlockHost H;
  const int d = L.box.dim;
  if (node_block(L, d, &H, err) < 0) return STFEM_ERR_STATE;
  block_apply_host(H, L, d, q, Dt, W, x, y);
  return STFEM_OK;
}

// ---------------------------------------------------------------- allocation-free smoothing
// Scratch of stfem_smooth_noalloc: one static array per device that loads the
// library.  Host code must not use the symbol as an address; its device
// address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[STFEM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call per device).
int noalloc_scratch(stfem_h h, unsigned char **out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != h->device) {
    h->err = "stfem_smooth_noalloc: the current device is not the handle's device";
    return STFEM_ERR_STATE;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    h->err = "stfem_smooth_noalloc: device index out of range";
    return STFEM_ERR_STATE;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
  return 0;
}

template <typename T>
int smooth_noalloc_t(stfem_h h, int level, const double *b, double *d, int nsw, int zero_init) {
  DLevel<T> &L = levels<T>(h)[level];
  // a level on the wide patch kernel also needs its slot results and ticket
  // counters
  const size_t wz = L.wide ? (size_t)L.sumC * sizeof(T) + (size_t)L.npatch * sizeof(int) : 0;
  // and a matrix-free level its per-cell results
  const size_t mz = mf_scratch_floats(L, h->q) * sizeof(T);
  const size_t need = (3 * (size_t)L.N + (size_t)L.sumC) * sizeof(T) + wz + mz;
  if (need > STFEM_NOALLOC_SCRATCH_BYTES) {
    h->err = "stfem_smooth_noalloc: level " + std::to_string(level) + " needs " + std::to_string(need) +
             " bytes of scratch, more than the " + std::to_string((size_t)STFEM_NOALLOC_SCRATCH_BYTES) +
             "-byte static array";
    return STFEM_ERR_ARG;
  }
  unsigned char *base = nullptr;
  CKR(noalloc_scratch(h, &base));
  // layout: b_T | d_T | r_T | y_T [| z_T | tickets] [| per-cell results]
  // (each 256-byte aligned)
  auto align = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t vb = align((size_t)L.N * sizeof(T));
  const size_t yb = align((size_t)L.sumC * sizeof(T));
  const size_t tb = align((size_t)L.npatch * sizeof(int));
  const size_t total = 3 * vb + (L.wide ? 2 * yb + tb : yb) + mz;
  if (total > STFEM_NOALLOC_SCRATCH_BYTES) {
    h->err = "stfem_smooth_noalloc: level does not fit the static array after alignment";
    return STFEM_ERR_ARG;
  }
  T *bT = reinterpret_cast<T *>(base);
  T *dT = reinterpret_cast<T *>(base + vb);
  T *rT = reinterpret_cast<T *>(base + 2 * vb);
  T *yT = reinterpret_cast<T *>(base + 3 * vb);
  T *zT = L.wide ? reinterpret_cast<T *>(base + 3 * vb + yb) : nullptr;
  int *tT = L.wide ? reinterpret_cast<int *>(base + 3 * vb + 2 * yb) : nullptr;
  T *mT = mz ? reinterpret_cast<T *>(base + 3 * vb + (L.wide ? 2 * yb + tb : yb)) : nullptr;
  const TimeCoef<T> tc = time_coef<T>(h->T, h->tau);
  cudaStream_t s = h->stream;
  // the array keeps the last call's contents: the tickets must start at zero
  if (tT) CK(cudaMemsetAsync(tT, 0, (size_t)L.npatch * sizeof(int), s));
  k_convert<double, T><<<grid_for(L.N, 256), 256, 0, s>>>(L.N, b, bT);
  if (!zero_init) k_convert<double, T><<<grid_for(L.N, 256), 256, 0, s>>>(L.N, d, dT);
  for (int it = 0; it < nsw; ++it) {
    const bool zero = zero_init && it == 0;
    const T *res = bT;
    if (!zero) {
      launch_spmv<T>(h, L, tc, dT, bT, rT, 1, 1, mT);
      res = rT;
    }
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (L.tc) { // the tensor-core apply that stfem_smooth uses on this level
        launch_patch_tc(h, L, res, yT, 1);
        done = true;
      }
    }
    if (!done) launch_patch_apply_to<T>(h, L, res, yT, zT, tT);
    k_vanka_update<T><<<grid_for(L.N, 256), 256, 0, s>>>(L.N, L.iptr, L.ipos, L.scale, yT, dT, zero ? 1 : 0, 1,
                                                         L.sumC);
  }
  k_convert<T, double><<<grid_for(L.N, 256), 256, 0, s>>>(L.N, dT, d);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  CKR(check_dev_err(h));
  return 0;
}

// Ring shape of the streaming patch apply of one V-cycle level: read, or pin
// (set != 0).  Only levels that run the streaming kernel have one.
template <typename T>
int stream_shape_io(stfem_h h, int level, int set, int *nst, int *per_sm, int *tile) {
  std::vector<DLevel<T>> &Ls = levels<T>(h);
  DLevel<T> &L = Ls[level];
  if (L.form != 1 || L.tc || L.wide || L.npatch == 0) {
    if (set) {
      h->err = "the level does not run the streaming patch apply";
      return STFEM_ERR_ARG;
    }
    *nst = *per_sm = *tile = 0;
    return STFEM_OK;
  }
  if (!set) {
    int threads, grid, n;
    size_t smem;
    stream_shape(h, L, &threads, &smem, &grid, &n);
    *nst = n;
    *per_sm = L.tune_nst > 0 ? L.tune_cap : (h->dim == 2 ? 5 : 3);
    *tile = std::max(1, L.tune_tile);
    return STFEM_OK;
  }
  if (*nst < 2 || *nst > STREAM_STAGES || *per_sm < 1 || *per_sm > 8 || *tile < 1 || *tile > 64) {
    h->err = "stream shape out of range (2 <= nst <= 12, 1 <= per_sm <= 8, 1 <= tile <= 64)";
    return STFEM_ERR_ARG;
  }
  const int o_nst = L.tune_nst, o_cap = L.tune_cap, o_tile = L.tune_tile;
  L.tune_nst = *nst;
  L.tune_cap = *per_sm;
  L.tune_tile = *tile;
  int threads, grid, n;
  size_t smem;
  stream_shape(h, L, &threads, &smem, &grid, &n);
  if (smem > 227u * 1024u) {
    L.tune_nst = o_nst;
    L.tune_cap = o_cap;
    L.tune_tile = o_tile;
    h->err = "stream shape needs more shared memory than a CTA has";
    return STFEM_ERR_ARG;
  }
  drop_graphs(h);
  return STFEM_OK;
}

int stream_shape_call(stfem_h h, int level, int set, int *nst, int *per_sm, int *tile) {
  if (!h || !nst || !per_sm || !tile) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  if (level < 1 || level >= h->nlev) {
    h->err = "level out of range (levels 1 .. n_levels-1 have patches)";
    return STFEM_ERR_ARG;
  }
  return h->precision == STFEM_MIXED ? stream_shape_io<float>(h, level, set, nst, per_sm, tile)
                                     : stream_shape_io<double>(h, level, set, nst, per_sm, tile);
}

// Shape of the tensor-core patch apply of one level: read, or pin (set != 0).
int tc_shape_call(stfem_h h, int level, int set, int *split, int *deep) {
  if (!h || !split || !deep) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  if (level < 1 || level >= h->nlev) {
    h->err = "level out of range (levels 1 .. n_levels-1 have patches)";
    return STFEM_ERR_ARG;
  }
  if (h->precision != STFEM_MIXED || !h->L32[level].tc) {
    if (set) {
      h->err = "the level does not run the tensor-core patch apply";
      return STFEM_ERR_ARG;
    }
    *split = *deep = -1;
    return STFEM_OK;
  }
  DLevel<float> &L = h->L32[level];
  if (!set) {
    *split = L.tc_split;
    *deep = L.tc_deep && L.tc_nst_deep > L.tc_nst ? 1 : 0;
    return STFEM_OK;
  }
  if ((*split != 0 && *split != 1) || (*deep != 0 && *deep != 1)) {
    h->err = "tensor-core shape out of range (split and deep are 0 or 1)";
    return STFEM_ERR_ARG;
  }
  if (*deep && L.tc_nst_deep <= L.tc_nst) {
    h->err = "no deeper ring fits next to this level's patches";
    return STFEM_ERR_ARG;
  }
  L.tc_split = *split;
  L.tc_deep = *deep;
  drop_graphs(h);
  return STFEM_OK;
}

} // namespace

// ============================================================ C ABI
extern "C" {

int stfem_setup(const stfem_mesh *mesh, const stfem_degrees *deg, const stfem_material *mat, const stfem_bcs *bcs,
                double tau, stfem_h *out) {
  if (!out) {
    g_setup_err = "null argument";
    return STFEM_ERR_ARG;
  }
  *out = nullptr;
  stfem_h h = new stfem_ctx();
  cudaGetDevice(&h->device);
  if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || h->nsm < 1 ||
      cudaDeviceGetAttribute(&h->clock_khz, cudaDevAttrClockRate, h->device) != cudaSuccess || h->clock_khz < 1) {
    h->err = "cannot query the device's multiprocessor count and clock";
    return fail_setup(h, STFEM_ERR_CUDA);
  }
  h->dot_blocks = 4 * h->nsm;
  {
    int rc0 = stfem::build_hierarchy(mesh, deg, mat, bcs, tau, &h->hl, &h->Pu, &h->Pp, &h->err);
    if (rc0 < 0) return fail_setup(h, rc0);
  }
  const int d = mesh->dim;
  const int pid = bcs->problem;
  h->dim = d;
  h->r = deg->r;
  h->k = deg->k;
  h->q = deg->k + 1;
  h->nlev = mesh->n_levels;
  h->tau = tau;
  h->t0 = bcs->t0;
  h->problem = pid;
  h->T = stfem::make_temporal(deg->k);
  // upload FP64 operators
  h->L64.resize(h->nlev);
  int rc;
  for (int l = 0; l < h->nlev; ++l) {
    if ((rc = upload_level_matrix(h, h->L64[l], h->hl[l], h->q)) < 0) return fail_setup(h, rc);
    if (l >= 1 && (rc = upload_transfer(h, h->L64[l], h->Pu[l], h->Pp[l])) < 0) return fail_setup(h, rc);
  }
  // geometry and problem of the finest level
  const stfem::Level &F = h->hl.back();
  GeomDev &g = h->geom;
  g.dim = d;
  g.r = h->r;
  for (int i = 0; i < 3; ++i) {
    g.lo[i] = F.box.lo[i];
    g.h[i] = F.box.h[i];
    g.n[i] = F.box.n[i];
    g.udims[i] = F.U.dims[i];
    g.pdims[i] = F.P.dims[i];
  }
  for (int i = 0; i < 8; ++i) {
    g.refU[i] = i < (int)F.U.ref.size() ? F.U.ref[i] : 0.0;
    g.refP[i] = i < (int)F.P.ref.size() ? F.P.ref[i] : 0.0;
  }
  h->prob.id = pid;
  h->prob.dim = d;
  h->prob.rho = mat->rho;
  h->prob.alpha = mat->alpha;
  h->prob.c0 = mat->c0;
  h->prob.b1 = deg->form == STFEM_FORM_PROBLEM_B_1 ? 1 : 0;
  h->prob.hF = F.box.hF;
  h->prob.gam_a = 5.0e4 * h->r * (h->r + 1);
  h->prob.gam_b = 0.5 * h->r * (h->r - 1);
  {
    bool neumann = false;
    for (int f = 0; f < 6; ++f) {
      h->prob.bc_u[f] = f < 2 * d ? bcs->bc_u[f] : 0;
      h->prob.bc_p[f] = f < 2 * d ? bcs->bc_p[f] : 0;
      neumann = neumann || h->prob.bc_u[f] != 0 || h->prob.bc_p[f] != 0;
    }
    // nonzero traces, or Neumann data of an exact solution
    h->prob.data = (pid == STFEM_PROBLEM_TRACE || (pid == STFEM_PROBLEM_SIN && neumann)) ? 1 : 0;
  }
  if ((rc = build_load_tables(h)) < 0) return fail_setup(h, rc);
  h->lt.top_neumann = (d == 3 && bcs->bc_u[5] == 1) ? 1 : 0;
  const long N = h->L64.back().N;
  if ((rc = dalloc(h, &h->w, N)) < 0 || (rc = dalloc(h, &h->rvec, N)) < 0 || (rc = dalloc(h, &h->zt, N)) < 0 ||
      (rc = dalloc(h, &h->rhs, N)) < 0 || (rc = dalloc(h, &h->xs, N)) < 0 ||
      (rc = dalloc(h, &h->ys, F.ns)) < 0 || (rc = dalloc(h, &h->hn2, 1)) < 0 ||
      (rc = dalloc(h, &h->src, (size_t)h->q * F.box.ncell * h->lt.nq * 4)) < 0 ||
      (rc = dalloc(h, &h->hnorm, 1)) < 0 || (rc = dalloc(h, &h->status, 4)) < 0 ||
      (rc = dalloc(h, &h->dev_err, 1)) < 0 ||
      (rc = dalloc(h, &h->partial, (size_t)h->dot_blocks * (MAXM + 1))) < 0 ||
      (rc = upload(h, &h->chi, h->T.chi_m1)) < 0 || (rc = upload(h, &h->tnode, h->T.t)) < 0)
    return fail_setup(h, rc);
  if (cudaHostAlloc((void **)&h->status_host, 4 * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
    h->err = "cudaHostAlloc failed";
    return fail_setup(h, STFEM_ERR_CUDA);
  }
  // uploads went through the legacy stream: wait for them there (no
  // device-wide synchronisation, which would also wait for, and can disturb
  // the graph captures of, handles run by other threads)
  if (cudaMemset(h->dev_err, 0, sizeof(int)) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) {
    h->err = "device error during setup";
    return fail_setup(h, STFEM_ERR_CUDA);
  }
  *out = h;
  return STFEM_OK;
}

int stfem_gmg_setup(stfem_h h, const stfem_gmg_params *p) {
  if (!h || !p) return STFEM_ERR_ARG;
  if (!(p->omega > 0.0) || p->n_sweeps < 1 || (p->precision != STFEM_FP64 && p->precision != STFEM_MIXED) ||
      p->patch_form < STFEM_PATCH_AUTO || p->patch_form > STFEM_PATCH_TIME_DIAGONAL ||
      (p->patch_kind != STFEM_PATCHES_VERTEX && p->patch_kind != STFEM_PATCHES_CELL) ||
      (p->update != STFEM_UPDATE_AVERAGE && p->update != STFEM_UPDATE_OVERWRITE) || p->n_rhs < 0 ||
      p->n_rhs > STFEM_MAX_RHS) {
    h->err = "invalid GMG parameters";
    return STFEM_ERR_ARG;
  }
  if (h->precision >= 0) {
    h->err = "stfem_gmg_setup may only be called once per handle";
    return STFEM_ERR_STATE;
  }
  h->omega = p->omega;
  h->nsweeps = p->n_sweeps;
  h->patch_kind = p->patch_kind;
  h->update = p->update;
  h->nrhs_cap = std::max(1, p->n_rhs);
  h->precision = p->precision;
  const bool mixed = p->precision == STFEM_MIXED;
  if (mixed) {
    h->L32.resize(h->nlev);
    for (int l = 0; l < h->nlev; ++l) {
      CKR(upload_level_matrix(h, h->L32[l], h->hl[l], h->q));
      if (l >= 1) CKR(upload_transfer(h, h->L32[l], h->Pu[l], h->Pp[l]));
    }
    CKR(upload_level_df(h, h->L64.back(), h->hl.back()));
    if (h->fine_op == STFEM_OPERATOR_MATRIX_FREE) {
      CKR(upload_matfree(h, h->L32.back(), h->hl.back()));
      h->L32.back().use_mf = h->L32.back().has_mf;
    }
  }
  int form = p->patch_form;
  if (form == STFEM_PATCH_AUTO) form = mixed ? STFEM_PATCH_TIME_DIAGONAL : STFEM_PATCH_DENSE;
  CKR(prepare_stream_kernels(h));
  stfem::TimeDiag td;
  if (form == STFEM_PATCH_TIME_DIAGONAL) {
    std::string err;
    if (!stfem::time_diag(h->T, h->tau, &td, &err)) {
      h->err = "time-diagonal patch form: " + err;
      return STFEM_ERR_STATE;
    }
  }
  // the coarse inverse (host, FP64) is computed while the patches are set up
  // (host extraction, device factorisation); nothing writes level 0 meanwhile,
  // and an early return waits for it in the future's destructor
  const int n0 = (int)(h->hl[0].ns * h->q);
  std::vector<double> A0;
  std::future<bool> coarse = std::async(std::launch::async, [&]() {
    A0 = stfem::dense_slab(h->hl[0], h->T, h->tau);
    return stfem::invert(A0.data(), n0);
  });
  // time-diagonal inverses are factorised on the device unless asked otherwise
  const bool dev_factor = form == STFEM_PATCH_TIME_DIAGONAL && !p->factor_host;
  for (int l = 1; l < h->nlev; ++l) {
    stfem::Patches P;
    std::string err;
    if (stfem::build_patches(h->hl[l], h->T, h->tau, mixed ? 4 : 2, &P, &err, !dev_factor,
                             form == STFEM_PATCH_TIME_DIAGONAL ? &td : nullptr, h->patch_kind) < 0) {
      h->err = err + " on level " + std::to_string(l);
      return STFEM_ERR_SINGULAR_PATCH;
    }
    if (mixed) {
      set_diag(h->L32[l], td);
      CKR(upload_patches(h, h->L32[l], P, h->omega, h->update));
      CKR(check_patch_shape(h, h->L32[l]));
      if (dev_factor) CKR(factor_on_device(h, h->L32[l], h->hl[l], P, td));
      if (h->nrhs_cap > 1 && form == STFEM_PATCH_TIME_DIAGONAL)
        CKR(dev_factor ? build_tc_tiles_device(h, h->L32[l], P) : upload_tc_tiles(h, h->L32[l], P));
    } else {
      set_diag(h->L64[l], td);
      CKR(upload_patches(h, h->L64[l], P, h->omega, h->update));
      CKR(check_patch_shape(h, h->L64[l]));
      if (dev_factor) CKR(factor_on_device(h, h->L64[l], h->hl[l], P, td));
    }
  }
  for (int l = 1; l < h->nlev; ++l) {
    if (mixed) {
      CKR(prepare_wide(h, h->L32[l]));
      CKR(autotune_stream(h, h->L32[l]));
    } else {
      CKR(prepare_wide(h, h->L64[l]));
      CKR(autotune_stream(h, h->L64[l]));
    }
  }
  CKR(check_dev_err(h));
  if (!coarse.get()) {
    h->err = "singular coarse matrix";
    return STFEM_ERR_SINGULAR_PATCH;
  }
  CKR(upload(h, &h->coarse_inv, A0));
  if (h->nrhs_cap > 1) {
    for (int l = 0; l < h->nlev; ++l) {
      if (mixed)
        CKR(ensure_columns(h, h->L32[l], h->nrhs_cap));
      else
        CKR(ensure_columns(h, h->L64[l], h->nrhs_cap));
    }
    if (mixed)
      for (int l = 1; l < h->nlev; ++l) CKR(autotune_tc(h, h->L32[l]));
    CKR(check_dev_err(h));
  }
  CK(cudaStreamSynchronize(0)); // uploads of the legacy stream (see stfem_setup)
  return STFEM_OK;
}

int stfem_set_stop(stfem_h h, int mode) {
  if (!h) return STFEM_ERR_ARG;
  if (mode != STFEM_STOP_RELATIVE && mode != STFEM_STOP_ABSOLUTE) {
    h->err = "unknown stopping rule";
    return STFEM_ERR_ARG;
  }
  h->stop = mode;
  return STFEM_OK;
}

int stfem_set_launch_cap(stfem_h h, int max_ctas) {
  if (!h || max_ctas < 0) return STFEM_ERR_ARG;
  if (max_ctas != h->launch_cap) drop_graphs(h);
  h->launch_cap = max_ctas;
  return STFEM_OK;
}

int stfem_get_stream_shape(stfem_h h, int level, int *nst, int *per_sm, int *tile) {
  return stream_shape_call(h, level, 0, nst, per_sm, tile);
}

int stfem_set_stream_shape(stfem_h h, int level, int nst, int per_sm, int tile) {
  return stream_shape_call(h, level, 1, &nst, &per_sm, &tile);
}

int stfem_get_tc_shape(stfem_h h, int level, int *split, int *deep) {
  return tc_shape_call(h, level, 0, split, deep);
}

int stfem_set_tc_shape(stfem_h h, int level, int split, int deep) {
  return tc_shape_call(h, level, 1, &split, &deep);
}

int stfem_set_fine_operator(stfem_h h, int choice) {
  if (!h || choice < STFEM_OPERATOR_AUTO || choice > STFEM_OPERATOR_MATRIX_FREE) {
    if (h) h->err = "unknown operator choice";
    return STFEM_ERR_ARG;
  }
  if (h->precision >= 0) {
    h->err = "stfem_set_fine_operator must be called before stfem_gmg_setup";
    return STFEM_ERR_STATE;
  }
  h->fine_op = choice;
  return STFEM_OK;
}

int stfem_set_patch_kernel(stfem_h h, int choice) {
  if (!h || choice < STFEM_PATCH_KERNEL_AUTO || choice > STFEM_PATCH_KERNEL_WIDE) {
    if (h) h->err = "unknown patch-apply kernel choice";
    return STFEM_ERR_ARG;
  }
  CKR(require_gmg(h));
  if (choice != h->patch_kernel) drop_graphs(h);
  h->patch_kernel = choice;
  for (int l = 1; l < h->nlev; ++l) {
    if (h->precision == STFEM_MIXED)
      CKR(prepare_wide(h, h->L32[l]));
    else
      CKR(prepare_wide(h, h->L64[l]));
  }
  CK(cudaStreamSynchronize(0)); // the ticket counters were cleared on the legacy stream
  return STFEM_OK;
}

int stfem_set_wait_limit(stfem_h h, double seconds) {
  if (!h || !(seconds > 0.0) || seconds > 60.0) {
    if (h) h->err = "wait limit must lie in (0, 60] seconds";
    return STFEM_ERR_ARG;
  }
  const long long cyc = std::max(1LL, (long long)(seconds * 1e3 * (double)h->clock_khz));
  if (cyc != h->wait_cycles) drop_graphs(h);
  h->wait_cycles = cyc;
  return STFEM_OK;
}

int stfem_stall_copies(stfem_h h, int on) {
  if (!h) return STFEM_ERR_ARG;
  if ((on != 0) != (h->stall_copies != 0)) drop_graphs(h);
  h->stall_copies = on != 0;
  return STFEM_OK;
}

int stfem_set_stream(stfem_h h, void *stream) {
  if (!h) return STFEM_ERR_ARG;
  h->stream = (cudaStream_t)stream;
  return STFEM_OK;
}

int stfem_level_info(stfem_h h, int level, long long *n_slab, long long *n_state, long long *n_patches,
                     long long *inv_bytes) {
  if (!h) return STFEM_ERR_ARG;
  if (level == -1) level = h->nlev - 1;
  CKR(check_level(h, level, false));
  const stfem::Level &L = h->hl[level];
  if (n_slab) *n_slab = L.ns * h->q;
  if (n_state) *n_state = L.ns;
  long long np = 0, ib = 0;
  if (h->precision == STFEM_MIXED && level >= 1) {
    np = h->L32[level].npatch;
    ib = h->L32[level].inv_elems * 4;
  } else if (h->precision == STFEM_FP64 && level >= 1) {
    np = h->L64[level].npatch;
    ib = h->L64[level].inv_elems * 8;
  }
  if (n_patches) *n_patches = np;
  if (inv_bytes) *inv_bytes = ib;
  return STFEM_OK;
}

int stfem_apply(stfem_h h, int level, const double *x, double *y) {
  if (!h || !x || !y) return STFEM_ERR_ARG;
  CKR(check_level(h, level, true));
  if (level == -1 || h->precision != STFEM_MIXED) return apply_t<double>(h, level == -1 ? h->nlev - 1 : level, x, y);
  return apply_t<float>(h, level, x, y);
}

int stfem_smooth(stfem_h h, int level, const double *b, double *d, int n_sweeps, int zero_init) {
  if (!h || !b || !d || n_sweeps < 1) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  CKR(check_level(h, level, false));
  if (level < 1) {
    h->err = "smoothing is defined on levels >= 1";
    return STFEM_ERR_ARG;
  }
  if (h->precision == STFEM_MIXED) return smooth_t<float>(h, level, b, d, n_sweeps, zero_init);
  return smooth_t<double>(h, level, b, d, n_sweeps, zero_init);
}

int stfem_smooth_batch(stfem_h h, int level, int n_rhs, const double *b, double *d, int n_sweeps, int zero_init) {
  if (!h || !b || !d || n_sweeps < 1) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  CKR(check_level(h, level, false));
  if (level < 1) {
    h->err = "smoothing is defined on levels >= 1";
    return STFEM_ERR_ARG;
  }
  if (n_rhs < 1 || n_rhs > h->nrhs_cap) {
    h->err = "n_rhs must be between 1 and the n_rhs given to stfem_gmg_setup";
    return STFEM_ERR_ARG;
  }
  if (h->precision == STFEM_MIXED) return smooth_t<float>(h, level, b, d, n_sweeps, zero_init, n_rhs);
  return smooth_t<double>(h, level, b, d, n_sweeps, zero_init, n_rhs);
}

int stfem_smooth_noalloc(stfem_h h, int level, const double *b, double *d, int n_sweeps, int zero_init) {
  if (!h || !b || !d || n_sweeps < 1) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  CKR(check_level(h, level, false));
  if (level < 1) {
    h->err = "smoothing is defined on levels >= 1";
    return STFEM_ERR_ARG;
  }
  if (h->prof) {
    h->err = "stfem_smooth_noalloc: turn profiling off first (it creates CUDA events)";
    return STFEM_ERR_STATE;
  }
  if (h->precision == STFEM_MIXED) return smooth_noalloc_t<float>(h, level, b, d, n_sweeps, zero_init);
  return smooth_noalloc_t<double>(h, level, b, d, n_sweeps, zero_init);
}

int stfem_restrict(stfem_h h, int level, const double *r_fine, double *b_coarse) {
  if (!h || !r_fine || !b_coarse) return STFEM_ERR_ARG;
  CKR(check_level(h, level, false));
  if (level < 1) return STFEM_ERR_ARG;
  if (h->precision == STFEM_MIXED) return transfer_t<float>(h, level, r_fine, b_coarse, true);
  return transfer_t<double>(h, level, r_fine, b_coarse, true);
}

int stfem_prolongate_add(stfem_h h, int level, const double *d_coarse, double *d_fine) {
  if (!h || !d_coarse || !d_fine) return STFEM_ERR_ARG;
  CKR(check_level(h, level, false));
  if (level < 1) return STFEM_ERR_ARG;
  if (h->precision == STFEM_MIXED) return transfer_t<float>(h, level, d_coarse, d_fine, false);
  return transfer_t<double>(h, level, d_coarse, d_fine, false);
}

int stfem_coarse_solve(stfem_h h, const double *b, double *x) {
  if (!h || !b || !x) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  coarse<double>(h, b, x);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return STFEM_OK;
}

int stfem_vcycle(stfem_h h, const double *b, double *d) {
  if (!h || !b || !d) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  CKR(precondition(h, b, d, nullptr));
  CK(cudaStreamSynchronize(h->stream));
  CKR(check_dev_err(h));
  return STFEM_OK;
}

int slab_solve(stfem_h h, const double *rhs, double *x, double tol, int restart, int max_it, int *iters,
               double *rel_res, double *abs_res) {
  if (!h || !rhs || !x || restart < 1 || max_it < 0 || !(tol >= 0.0)) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  int it = 0;
  double rr = 0.0, ra = 0.0;
  int rc = fgmres(h, rhs, x, tol, restart, max_it, &it, &rr, &ra);
  if (iters) *iters = it;
  if (rel_res) *rel_res = rr;
  if (abs_res) *abs_res = ra;
  CKR(check_dev_err(h));
  return rc;
}

int slab_solve_batch(stfem_h h, int n_rhs, const double *rhs, double *x, double tol, int restart, int max_it,
                     int *iters_host, double *rel_res_host) {
  if (!h || !rhs || !x || !iters_host || !rel_res_host || restart < 1 || max_it < 0 || !(tol >= 0.0))
    return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  if (n_rhs < 1 || n_rhs > h->nrhs_cap) {
    h->err = "n_rhs must be between 1 and the n_rhs given to stfem_gmg_setup";
    return STFEM_ERR_ARG;
  }
  const int rc = fgmres_batch(h, n_rhs, rhs, x, tol, restart, max_it, iters_host, rel_res_host);
  CK(cudaStreamSynchronize(h->stream));
  CKR(check_dev_err(h));
  return rc;
}

int stfem_apply_krylov(stfem_h h, const double *x, double *y) {
  if (!h || !x || !y) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  DLevel<double> &F = h->L64.back();
  const TimeCoef<double> tc = time_coef<double>(h->T, h->tau);
  if (h->precision == STFEM_MIXED && F.has_df) {
    float *xf = h->L32.back().b; // V-cycle input buffer, free between calls
    {
      Launch G_(h, STFEM_KCLASS_OTHER, F.N * 12.0, 0.0);
      k_convert<double, float><<<grid_for(F.N, 256), 256, 0, h->stream>>>(F.N, x, xf);
    }
    launch_spmv_df(h, F, tc, xf, y);
  } else {
    launch_spmv<double>(h, F, tc, x, nullptr, y, 0);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return STFEM_OK;
}

int stfem_vcycle_batch(stfem_h h, int n_rhs, const double *b, double *d) {
  if (!h || !b || !d) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  if (n_rhs < 1 || n_rhs > h->nrhs_cap) {
    h->err = "n_rhs must be between 1 and the n_rhs given to stfem_gmg_setup";
    return STFEM_ERR_ARG;
  }
  const int L = h->nlev - 1;
  const long N = h->L64.back().N;
  const int nbk = grid_for(N, 256);
  cudaStream_t s = h->stream;
  if (h->precision == STFEM_FP64) {
    DLevel<double> &G = h->L64[L];
    CK(cudaMemcpyAsync(G.b, b, (size_t)n_rhs * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    vcycle<double>(h, L, n_rhs);
    CK(cudaMemcpyAsync(d, G.d, (size_t)n_rhs * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    DLevel<float> &G = h->L32[L];
    {
      Launch G_(h, STFEM_KCLASS_OTHER, N * 12.0 * n_rhs, 0.0);
      k_copy_cols<double, float><<<nbk * n_rhs, 256, 0, s>>>(N, n_rhs, b, N, G.b, N);
    }
    vcycle<float>(h, L, n_rhs);
    {
      Launch G_(h, STFEM_KCLASS_OTHER, N * 12.0 * n_rhs, 0.0);
      k_copy_cols<float, double><<<nbk * n_rhs, 256, 0, s>>>(N, n_rhs, G.d, N, d, N);
    }
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  CKR(check_dev_err(h));
  return STFEM_OK;
}

int stfem_solve_history(stfem_h h, double *hist_host, int cap, int *n) {
  if (!h || !n) return STFEM_ERR_ARG;
  int m = std::min<int>(cap, (int)h->hist.size());
  for (int i = 0; i < m && hist_host; ++i) hist_host[i] = h->hist[i];
  *n = m;
  return STFEM_OK;
}

int stfem_initial_state_at(stfem_h h, double t, double *state) {
  if (!h || !state) return STFEM_ERR_ARG;
  const stfem::Level &F = h->hl.back();
  {
    Launch G_(h, STFEM_KCLASS_OTHER, F.ns * 8.0, 0.0);
    k_interp<<<grid_for(F.ns, 256), 256, 0, h->stream>>>(h->geom, h->prob, h->lt, t, F.R, F.S, state);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return STFEM_OK;
}

int stfem_initial_state(stfem_h h, double *state) { return stfem_initial_state_at(h, h ? h->t0 : 0.0, state); }

static int slab_rhs_async(stfem_h h, int slab, const double *prev, double *rhs, double t0) {
  DLevel<double> &F = h->L64.back();
  const stfem::Level &HF = h->hl.back();
  TimeCoef<double> one{};
  one.q = 1;
  one.Dt[0] = 1.0;
  one.W[0] = 0.0;
  if (F.nb.pcouple) {
    // Problem B.1: the pressure row couples to the previous state through
    // c0 Mp P^- + alpha <div u^-, xi>, i.e. the volume part of -C alone (the
    // data term -alpha <u_D . n, xi> is added by k_rhs_data); the launch
    // takes its arguments by value, so the swap lasts for it alone
    if (!F.pu_cvol) {
      h->err = "Problem B.1 needs the volume coupling of the finest level";
      return STFEM_ERR_STATE;
    }
    const double *pu_c = F.nb.pu_c;
    F.nb.pu_c = F.pu_cvol;
    launch_spmv<double>(h, F, one, prev, nullptr, h->ys, 0);
    F.nb.pu_c = pu_c;
  } else {
    launch_spmv<double>(h, F, one, prev, nullptr, h->ys, 0); // S1 * state
  }
  const TimeCoef<double> tc = time_coef<double>(h->T, h->tau);
  const double t_prev = t0 + slab * h->tau;
  const long ncell = HF.box.ncell;
  const long nsrc = (long)h->q * ncell * h->lt.nq;
  if (h->prob.id != STFEM_PROBLEM_NONE) {
    Launch G_(h, STFEM_KCLASS_RHS, (double)nsrc * 32.0, 0.0);
    k_src_eval<<<grid_for(nsrc, 128), 128, 0, h->stream>>>(h->geom, h->prob, h->lt, h->q, h->tnode, t_prev, h->tau,
                                                           ncell, h->src);
  }
  {
    Launch G_(h, STFEM_KCLASS_RHS, (double)F.N * 16.0 + (double)nsrc * 32.0, 0.0);
    k_rhs<<<grid_for(F.N, 128), 128, 0, h->stream>>>(h->geom, h->prob, h->lt, h->q, tc, h->chi, h->tnode, t_prev,
                                                     h->tau, HF.R, HF.S, h->src, h->ys, rhs);
  }
  if (h->prob.data) {
    const long nrow = (long)h->q * (HF.R + HF.S);
    Launch G2_(h, STFEM_KCLASS_RHS, (double)nrow * 16.0, 0.0);
    k_rhs_data<<<grid_for(nrow, 128), 128, 0, h->stream>>>(h->geom, h->prob, h->lt, h->q, tc, h->chi, h->tnode,
                                                           t_prev, h->tau, HF.R, HF.S, rhs);
  }
  CK(cudaGetLastError());
  return 0;
}

int stfem_slab_rhs(stfem_h h, int slab, const double *prev_state, double *rhs) {
  if (!h || !prev_state || !rhs || slab < 0) return STFEM_ERR_ARG;
  CKR(slab_rhs_async(h, slab, prev_state, rhs, h->t0));
  CK(cudaStreamSynchronize(h->stream));
  return STFEM_OK;
}

int march(stfem_h h, int first_slab, int n_slabs, double *state, double tol, int restart, int max_it,
          int *iters_host) {
  if (!h || !state || n_slabs < 0 || first_slab < 0) return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  DLevel<double> &F = h->L64.back();
  int worst = STFEM_OK;
  for (int n = 0; n < n_slabs; ++n) {
    CKR(slab_rhs_async(h, first_slab + n, state, h->rhs, h->t0));
    {
      Launch G_(h, STFEM_KCLASS_OTHER, F.N * 8.0 + F.ns * 8.0, 0.0);
      k_repeat<<<grid_for(F.N, 256), 256, 0, h->stream>>>(F.ns, h->q, state, h->xs);
    }
    int it = 0;
    double rr = 0.0, ra = 0.0;
    int rc = fgmres(h, h->rhs, h->xs, tol, restart, max_it, &it, &rr, &ra);
    if (iters_host) iters_host[n] = it;
    if (rc < 0) return rc;
    if (rc > worst) worst = rc;
    CK(cudaMemcpyAsync(state, h->xs + (long)(h->q - 1) * F.ns, F.ns * sizeof(double), cudaMemcpyDeviceToDevice,
                       h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  CKR(check_dev_err(h));
  return worst;
}

int march_batch(stfem_h h, int n_rhs, const double *t0_host, int first_slab, int n_slabs, double *state,
                double tol, int restart, int max_it, int *iters_host) {
  if (!h || !t0_host || !state || n_slabs < 0 || first_slab < 0 || restart < 1 || max_it < 0 || !(tol >= 0.0))
    return STFEM_ERR_ARG;
  CKR(require_gmg(h));
  if (n_rhs < 1 || n_rhs > h->nrhs_cap) {
    h->err = "n_rhs must be between 1 and the n_rhs given to stfem_gmg_setup";
    return STFEM_ERR_ARG;
  }
  CKR(ensure_batch_workspace(h, restart));
  stfem_ctx::Batch &B = h->bt;
  DLevel<double> &F = h->L64.back();
  int worst = STFEM_OK;
  std::vector<int> it(n_rhs);
  std::vector<double> rr(n_rhs);
  for (int n = 0; n < n_slabs; ++n) {
    for (int c = 0; c < n_rhs; ++c) {
      double *st = state + (long)c * F.ns;
      CKR(slab_rhs_async(h, first_slab + n, st, B.rhs + (long)c * F.N, t0_host[c]));
      Launch G_(h, STFEM_KCLASS_OTHER, F.N * 8.0 + F.ns * 8.0, 0.0);
      k_repeat<<<grid_for(F.N, 256), 256, 0, h->stream>>>(F.ns, h->q, st, B.xs + (long)c * F.N);
    }
    const int rc = fgmres_batch(h, n_rhs, B.rhs, B.xs, tol, restart, max_it, it.data(), rr.data());
    if (iters_host)
      for (int c = 0; c < n_rhs; ++c) iters_host[(long)n * n_rhs + c] = it[c];
    if (rc < 0) return rc;
    if (rc > worst) worst = rc;
    for (int c = 0; c < n_rhs; ++c)
      CK(cudaMemcpyAsync(state + (long)c * F.ns, B.xs + (long)c * F.N + (long)(h->q - 1) * F.ns,
                         F.ns * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  CKR(check_dev_err(h));
  return worst;
}

int stfem_profile(stfem_h h, int enable) {
  if (!h) return STFEM_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  h->prof = enable != 0;
  for (auto &k : h->kstat) k = stfem_ctx::KStat();
  h->pending.clear();
  h->evnext = 0;
  return STFEM_OK;
}

int stfem_profile_read(stfem_h h, int kclass, long long *launches, double *ms, double *bytes, double *flops) {
  if (!h || kclass < 0 || kclass >= STFEM_KCLASS_COUNT) return STFEM_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  // resolve recorded event pairs into per-class times
  for (const auto &pe : h->pending) {
    float t = 0.f;
    if (pe.second + 1 < h->evnext &&
        cudaEventElapsedTime(&t, h->evpool[pe.second], h->evpool[pe.second + 1]) == cudaSuccess)
      h->kstat[pe.first].ms += t;
  }
  h->pending.clear();
  h->evnext = 0;
  const auto &k = h->kstat[kclass];
  if (launches) *launches = k.launches;
  if (ms) *ms = k.ms;
  if (bytes) *bytes = k.bytes;
  if (flops) *flops = k.flops;
  return STFEM_OK;
}

int stfem_footprint_bytes(stfem_h h, long long *bytes) {
  if (!h || !bytes) return STFEM_ERR_ARG;
  *bytes = h->device_bytes;
  return STFEM_OK;
}

int stfem_launch_count(stfem_h h, long long *n) {
  if (!h || !n) return STFEM_ERR_ARG;
  *n = h->launches;
  return STFEM_OK;
}

const char *stfem_last_error(stfem_h h) { return h ? h->err.c_str() : g_setup_err.c_str(); }

void stfem_destroy(stfem_h h) {
  if (!h) return;
  // every entry point has synchronised its stream before returning; cudaFree
  // waits for the device work that may still use the memory
  for (void *p : h->allocs) cudaFree(p);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  for (auto &g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto &g : h->bt.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->status_host) cudaFreeHost(h->status_host);
  if (h->bt.host) cudaFreeHost(h->bt.host);
  if (h->grp_ev) cudaEventDestroy(h->grp_ev);
  delete h;
}

} // extern "C"

// ============================================================ groups of handles
// Several handles (problems of different meshes, degrees, materials: uneven
// instances) advanced in lockstep, one FGMRES step per member per group step,
// with the patch applies of each V-cycle stage fused across members: one
// launch of the streaming (or wide) patch kernel takes the patches of every
// member at that stage from a job table.  Every other kernel of a member runs
// on the member's own stream, as in the single-handle path; the fused launch
// runs on the group's stream between events, so members still overlap.  A
// member's arithmetic is the single-handle path's: the same kernels in the
// same order, a patch computed the same way in any launch.

namespace {

struct GroupMember {
  stfem_h h = nullptr;
  long long id = 0;
  int first = 0, n_slabs = 0, slab = 0;
  double *state = nullptr; // device, n_state
  double tol = 1e-8;
  int restart = 30, max_it = 500;
  // FGMRES state of the current slab solve
  enum Phase { START, INIT, ITER, FIN, DONE } phase = START;
  int j = 0, it = 0, jlast = -1;
  double beta0 = 0.0, bound = 0.0, beta = 0.0;
  int status = STFEM_OK;
  std::vector<int> iters;
  std::vector<double> slab_ms;
  std::chrono::steady_clock::time_point t_slab;
  cudaEvent_t ev = nullptr;
};

// Fused launch shapes picked by timing (ring stages, CTAs per SM, patch tile),
// keyed by the precision, the time nodes, the largest patch and the patch
// count (in powers of two): the candidates only spread patches differently
// over CTAs, so the choice never changes a result.
struct GroupTune {
  std::map<std::tuple<int, int, int, int>, std::array<int, 3>> shape;
};

} // namespace

struct stfem_group_ctx {
  std::string err;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  long long next_id = 1;
  std::vector<std::unique_ptr<GroupMember>> members;
  GroupTune tune;
  long long fused_launches = 0, fused_jobs = 0;
};

namespace {

// Patch applies of one V-cycle stage for a set of (member, level, input)
// items: time-diagonal levels are fused into job tables (streaming and wide
// kernels apart, at most MAXJOBS levels per launch); other levels (dense
// inverses, tensor-core levels) are applied on the member's stream.
template <typename T, int Q>
int fused_stage_q(stfem_group g, const std::vector<std::pair<stfem_h, int>> &items, bool use_r) {
  std::vector<std::pair<stfem_h, int>> stream_items, wide_items;
  for (const auto &it : items) {
    DLevel<T> &L = levels<T>(it.first)[it.second];
    const T *res = use_r ? L.r : L.b;
    if (L.form == 1 && !L.tc && L.wide)
      wide_items.push_back(it);
    else if (L.form == 1 && !L.tc)
      stream_items.push_back(it);
    else
      launch_patch_apply<T>(it.first, L, res);
  }
  auto join_in = [&](const std::vector<std::pair<stfem_h, int>> &v, size_t a, size_t b) -> int {
    for (size_t i = a; i < b; ++i) {
      stfem_h h = v[i].first;
      if (cudaEventRecord(h->grp_ev, h->stream) != cudaSuccess ||
          cudaStreamWaitEvent(g->stream, h->grp_ev, 0) != cudaSuccess) {
        g->err = "event record/wait failed";
        return STFEM_ERR_CUDA;
      }
    }
    return 0;
  };
  auto join_out = [&](const std::vector<std::pair<stfem_h, int>> &v, size_t a, size_t b) -> int {
    if (cudaEventRecord(g->ev, g->stream) != cudaSuccess) {
      g->err = "event record failed";
      return STFEM_ERR_CUDA;
    }
    for (size_t i = a; i < b; ++i)
      if (cudaStreamWaitEvent(v[i].first->stream, g->ev, 0) != cudaSuccess) {
        g->err = "stream wait failed";
        return STFEM_ERR_CUDA;
      }
    return 0;
  };
  for (size_t a = 0; a < stream_items.size(); a += MAXJOBS) {
    const size_t b = std::min(stream_items.size(), a + MAXJOBS);
    PatchJobs<T, MAXJOBS> J;
    J.njobs = 0;
    int maxCs = 0, nst = 0, cap = 0, tile = 1;
    size_t smem = 0;
    double bytes = 0.0, flops = 0.0;
    for (size_t i = a; i < b; ++i) {
      stfem_h h = stream_items[i].first;
      DLevel<T> &L = levels<T>(h)[stream_items[i].second];
      add_job(J, L, use_r ? L.r : L.b, L.ybuf);
      maxCs = std::max(maxCs, L.maxCs);
      bytes += L.patch_bytes;
      flops += L.patch_flops;
      h->launches++;
      h->kstat[STFEM_KCLASS_PATCH_APPLY].launches++;
      h->kstat[STFEM_KCLASS_PATCH_APPLY].bytes += L.patch_bytes;
      h->kstat[STFEM_KCLASS_PATCH_APPLY].flops += L.patch_flops;
    }
    const long total = J.first[J.njobs];
    // launch shape: the largest level's autotuned ring, or the group's own
    // tuning of this kind of stage
    stfem_h h0 = stream_items[a].first;
    const int dim = h0->dim;
    constexpr int VEC = Vec16<T>::n;
    int rows = 0;
    for (size_t i = a; i < b; ++i) {
      const DLevel<T> &L = levels<T>(stream_items[i].first)[stream_items[i].second];
      rows = std::max(rows, L.dc.nr * ((L.maxCs + VEC - 1) / VEC) + L.dc.nc * ((L.maxCs + VEC / 2 - 1) / (VEC / 2)));
    }
    const int nwc = std::max(1, (rows + 31) / 32);
    const int threads = 32 * (nwc + 1);
    int lg = 0;
    while ((1L << lg) < total) ++lg;
    const auto key = std::make_tuple((int)sizeof(T), Q, maxCs, lg);
    auto shape_of = [&](int st, int cp, int tl, size_t *sm, int *grid) {
      *sm = (size_t)stream_header(st) + (size_t)(Q + 2 * Q) * maxCs * sizeof(T);
      const int per_sm = std::max(1, std::min(cp, (int)((227u * 1024u) / *sm)));
      *grid = (int)std::min<long>((total + tl - 1) / tl, (long)h0->nsm * per_sm);
    };
    CKR(join_in(stream_items, a, b));
    auto found = g->tune.shape.find(key);
    if (found == g->tune.shape.end()) {
      static const int cand[][3] = STREAM_SHAPE_CANDIDATES;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best = 1e30f;
      std::array<int, 3> pick = {dim == 2 ? 2 : 4, dim == 2 ? 5 : 3, 1};
      for (const auto &c : cand) {
        int grid;
        shape_of(c[0], c[1], c[2], &smem, &grid);
        if (smem > 227u * 1024u) continue;
        cudaEventRecord(e0, g->stream);
        for (int t = 0; t < 3; ++t)
          k_patch_apply_stream<T, Q, MAXJOBS><<<grid, threads, smem, g->stream>>>(
              J, maxCs, c[2], h0->dev_err, c[0], h0->wait_cycles, h0->stall_copies);
        cudaEventRecord(e1, g->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          pick = {c[0], c[1], c[2]};
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      found = g->tune.shape.emplace(key, pick).first;
    }
    nst = found->second[0];
    cap = found->second[1];
    tile = found->second[2];
    int grid;
    shape_of(nst, cap, tile, &smem, &grid);
    if (smem > 227u * 1024u) {
      g->err = "fused patch apply: patches too large for the streaming kernel";
      return STFEM_ERR_ARG;
    }
    k_patch_apply_stream<T, Q, MAXJOBS><<<grid, threads, smem, g->stream>>>(J, maxCs, tile, h0->dev_err, nst,
                                                                          h0->wait_cycles, h0->stall_copies);
    g->fused_launches++;
    g->fused_jobs += J.njobs;
    (void)bytes;
    (void)flops;
    CKR(join_out(stream_items, a, b));
  }
  for (size_t a = 0; a < wide_items.size(); a += MAXJOBS) {
    const size_t b = std::min(wide_items.size(), a + MAXJOBS);
    PatchJobs<T, MAXJOBS> J;
    J.njobs = 0;
    size_t smem = 0;
    long ctas = 0;
    for (size_t i = a; i < b; ++i) {
      stfem_h h = wide_items[i].first;
      DLevel<T> &L = levels<T>(h)[wide_items[i].second];
      add_job(J, L, use_r ? L.r : L.b, L.ybuf, L.zbuf, L.ticket);
      smem = std::max(smem, wide_smem<T>(L, Q));
      ctas += L.npatch * (L.dc.nr + L.dc.nc);
      h->launches++;
      h->kstat[STFEM_KCLASS_PATCH_APPLY].launches++;
      h->kstat[STFEM_KCLASS_PATCH_APPLY].bytes += L.patch_bytes;
      h->kstat[STFEM_KCLASS_PATCH_APPLY].flops += L.patch_flops;
    }
    CKR(join_in(wide_items, a, b));
    k_patch_apply_wide<T, Q, PatchJobs<T, MAXJOBS>><<<(unsigned)ctas, WIDE_THREADS, smem, g->stream>>>(J);
    g->fused_launches++;
    g->fused_jobs += J.njobs;
    CKR(join_out(wide_items, a, b));
  }
  if (cudaGetLastError() != cudaSuccess) {
    g->err = "fused patch apply launch failed";
    return STFEM_ERR_CUDA;
  }
  return 0;
}

template <typename T>
int fused_stage(stfem_group g, int q, const std::vector<std::pair<stfem_h, int>> &items, bool use_r) {
  if (items.empty()) return 0;
  switch (q) {
  case 1: return fused_stage_q<T, 1>(g, items, use_r);
  case 2: return fused_stage_q<T, 2>(g, items, use_r);
  case 3: return fused_stage_q<T, 3>(g, items, use_r);
  case 4: return fused_stage_q<T, 4>(g, items, use_r);
  default: return fused_stage_q<T, 5>(g, items, use_r);
  }
}

// One V-cycle (from d = 0 on each member's finest level) for every handle of
// hs, stage by stage from the top: stage k smooths level nlev - 1 - k of each
// member that has it.  Per member the kernels and their order are those of
// vcycle(); the patch applies of a stage are fused.
template <typename T>
int group_vcycle(stfem_group g, const std::vector<stfem_h> &hs) {
  int K = 0, S = 0;
  for (stfem_h h : hs) {
    K = std::max(K, h->nlev - 1);
    S = std::max(S, h->nsweeps);
  }
  const int q = hs.empty() ? 1 : hs[0]->q;
  auto smooth_stage = [&](int k, bool pre) -> int {
    for (int sw = 0; sw < S; ++sw) {
      std::vector<std::pair<stfem_h, int>> items;
      for (stfem_h h : hs) {
        const int l = h->nlev - 1 - k;
        if (l < 1 || sw >= h->nsweeps) continue;
        DLevel<T> &L = levels<T>(h)[l];
        const bool zero = pre && sw == 0;
        if (!zero) launch_spmv<T>(h, L, time_coef<T>(h->T, h->tau), L.d, L.b, L.r, 1);
        items.push_back({h, l});
      }
      CKR(fused_stage<T>(g, q, items, !(pre && sw == 0)));
      for (const auto &it : items) {
        stfem_h h = it.first;
        DLevel<T> &L = levels<T>(h)[it.second];
        const bool zero = pre && sw == 0;
        Launch G_(h, STFEM_KCLASS_UPDATE, (double)L.N * (4.0 + 3.0 * sizeof(T)) + (double)L.sumC * (4.0 + sizeof(T)),
                  (double)L.sumC + 2.0 * L.N);
        k_vanka_update<T><<<grid_for(L.N, 256), 256, 0, h->stream>>>(L.N, L.iptr, L.ipos, L.scale, L.ybuf, L.d,
                                                                      zero ? 1 : 0, 1, L.sumC);
      }
    }
    return 0;
  };
  for (int k = 0; k < K; ++k) {
    CKR(smooth_stage(k, true));
    for (stfem_h h : hs) {
      const int l = h->nlev - 1 - k;
      if (l < 1) continue;
      std::vector<DLevel<T>> &Ls = levels<T>(h);
      DLevel<T> &L = Ls[l];
      launch_spmv<T>(h, L, time_coef<T>(h->T, h->tau), L.d, L.b, L.r, 1);
      restrict_to<T>(h, l, L.r, Ls[l - 1].b);
      if (l - 1 == 0) coarse<T>(h, Ls[0].b, Ls[0].d);
    }
  }
  for (stfem_h h : hs)
    if (h->nlev == 1) coarse<T>(h, levels<T>(h)[0].b, levels<T>(h)[0].d);
  for (int k = K - 1; k >= 0; --k) {
    for (stfem_h h : hs) {
      const int l = h->nlev - 1 - k;
      if (l < 1) continue;
      std::vector<DLevel<T>> &Ls = levels<T>(h);
      prolongate_add<T>(h, l, Ls[l - 1].d, Ls[l].d);
    }
    CKR(smooth_stage(k, false));
  }
  return 0;
}

// Enqueues the start of member m's next slab: right-hand side, initial guess
// (the previous end state at every time node) and the initial residual norm.
int member_start(GroupMember &m) {
  stfem_h h = m.h;
  DLevel<double> &F = h->L64.back();
  const long N = F.N;
  m.t_slab = std::chrono::steady_clock::now();
  CKR(ensure_workspace(h, m.restart));
  CKR(slab_rhs_async(h, m.first + m.slab, m.state, h->rhs, h->t0));
  {
    Launch G_(h, STFEM_KCLASS_OTHER, F.N * 8.0 + F.ns * 8.0, 0.0);
    k_repeat<<<grid_for(F.N, 256), 256, 0, h->stream>>>(F.ns, h->q, m.state, h->xs);
  }
  h->hist.clear();
  launch_spmv<double>(h, F, time_coef<double>(h->T, h->tau), h->xs, h->rhs, h->rvec, 1);
  multidot(h, 1, h->rvec, N, h->rvec, N, h->hn2);
  CK(cudaMemcpyAsync(h->status_host + 2, h->hn2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  m.phase = GroupMember::INIT;
  return 0;
}

// Enqueues the start of a restart cycle (v_0 = r / beta, g = beta e_1).
void member_cycle(GroupMember &m) {
  stfem_h h = m.h;
  const long N = h->L64.back().N;
  {
    Launch G_(h, STFEM_KCLASS_BLAS1, N * 16.0, (double)N);
    k_div<<<grid_for(N, 256), 256, 0, h->stream>>>(N, h->rvec, h->V, nullptr, m.beta);
  }
  {
    Launch G_(h, STFEM_KCLASS_OTHER, 8.0, 0.0);
    k_set<<<1, 1, 0, h->stream>>>(h->g, m.beta);
  }
  m.j = 0;
  m.jlast = -1;
}

// Enqueues the end of a cycle: y from the triangular system, x += Z y, and the
// true residual norm.
int member_finish(GroupMember &m) {
  stfem_h h = m.h;
  DLevel<double> &F = h->L64.back();
  const long N = F.N;
  const int kk = m.jlast + 1, m1 = m.restart + 1;
  cudaStream_t s = h->stream;
  {
    Launch G_(h, STFEM_KCLASS_OTHER, (double)kk * kk * 8.0, (double)kk * kk);
    k_backsolve<<<1, 1, 0, s>>>(kk, m1, h->H, h->g, h->y);
  }
  {
    Launch G_(h, STFEM_KCLASS_BLAS1, (double)N * (16.0 + kk * (h->precision == STFEM_FP64 ? 8.0 : 4.0)),
              2.0 * kk * N);
    if (h->precision == STFEM_FP64)
      k_update_x<double><<<grid_for(N, 256), 256, 0, s>>>(N, kk, h->Zd, N, h->y, h->xs);
    else
      k_update_x<float><<<grid_for(N, 256), 256, 0, s>>>(N, kk, h->Zf, N, h->y, h->xs);
  }
  launch_spmv<double>(h, F, time_coef<double>(h->T, h->tau), h->xs, h->rhs, h->rvec, 1);
  multidot(h, 1, h->rvec, N, h->rvec, N, h->hn2);
  CK(cudaMemcpyAsync(h->status_host + 2, h->hn2, sizeof(double), cudaMemcpyDeviceToHost, s));
  m.phase = GroupMember::FIN;
  return 0;
}

// The slab converged (or ran out of iterations): keep its end state, move on.
int member_next_slab(GroupMember &m, int rc) {
  stfem_h h = m.h;
  DLevel<double> &F = h->L64.back();
  CK(cudaMemcpyAsync(m.state, h->xs + (long)(h->q - 1) * F.ns, F.ns * sizeof(double), cudaMemcpyDeviceToDevice,
                     h->stream));
  m.iters.push_back(m.it);
  m.slab_ms.push_back(
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - m.t_slab).count());
  m.status = std::max(m.status, rc);
  ++m.slab;
  m.phase = m.slab < m.n_slabs ? GroupMember::START : GroupMember::DONE;
  return 0;
}

// One step of every member: members at the start of a slab or at the end of
// a cycle enqueue that work, the iterating members one FGMRES iteration with
// a shared, fused V-cycle; then every member's stream is synchronised once
// and each member's host state advances as in fgmres() and march().
int group_step(stfem_group g) {
  std::vector<GroupMember *> live;
  for (auto &up : g->members)
    if (up->phase != GroupMember::DONE && up->status >= 0) live.push_back(up.get());
  if (live.empty()) return 0;
  for (GroupMember *m : live)
    if (m->phase == GroupMember::START) {
      const int rc = member_start(*m);
      if (rc < 0) {
        m->status = rc;
        m->phase = GroupMember::DONE;
      }
    }
  std::vector<GroupMember *> iter;
  for (GroupMember *m : live)
    if (m->phase == GroupMember::ITER) iter.push_back(m);
  if (!iter.empty()) {
    std::vector<stfem_h> hs;
    for (GroupMember *m : iter) {
      CKR(iter_pre(m->h, m->j));
      hs.push_back(m->h);
    }
    const int rc = iter[0]->h->precision == STFEM_FP64 ? group_vcycle<double>(g, hs) : group_vcycle<float>(g, hs);
    if (rc < 0) return rc;
    for (GroupMember *m : iter) CKR(iter_post(m->h, m->j, m->restart + 1));
  }
  for (GroupMember *m : live)
    if (cudaStreamSynchronize(m->h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      g->err = "device error in a group step";
      return STFEM_ERR_CUDA;
    }
  for (GroupMember *m : live) {
    stfem_h h = m->h;
    if (m->phase == GroupMember::INIT) {
      const double beta0 = std::sqrt(h->status_host[2]);
      h->hist.push_back(1.0);
      m->it = 0;
      if (!std::isfinite(beta0)) {
        h->err = "initial residual is not finite";
        m->status = STFEM_ERR_BREAKDOWN;
        m->phase = GroupMember::DONE;
        continue;
      }
      m->beta0 = beta0;
      m->bound = h->stop == STFEM_STOP_ABSOLUTE ? m->tol : m->tol * beta0;
      if (beta0 == 0.0 || beta0 <= m->bound) {
        CKR(member_next_slab(*m, STFEM_OK));
        continue;
      }
      m->beta = beta0;
      member_cycle(*m);
      m->phase = GroupMember::ITER;
    } else if (m->phase == GroupMember::ITER) {
      const double res = h->status_host[0], hn = h->status_host[1];
      if (!std::isfinite(res) || !std::isfinite(hn)) {
        h->err = "FGMRES breakdown: non-finite Hessenberg entry";
        m->status = STFEM_ERR_BREAKDOWN;
        m->phase = GroupMember::DONE;
        continue;
      }
      ++m->it;
      m->jlast = m->j;
      h->hist.push_back(res / m->beta0);
      if (res <= m->bound || m->it >= m->max_it || hn == 0.0 || m->j + 1 >= m->restart)
        CKR(member_finish(*m));
      else
        ++m->j;
    } else if (m->phase == GroupMember::FIN) {
      const double res = std::sqrt(h->status_host[2]);
      if (!std::isfinite(res)) {
        h->err = "FGMRES breakdown: non-finite residual";
        m->status = STFEM_ERR_BREAKDOWN;
        m->phase = GroupMember::DONE;
        continue;
      }
      if (res <= m->bound) {
        CKR(member_next_slab(*m, STFEM_OK));
      } else if (m->it >= m->max_it) {
        CKR(member_next_slab(*m, STFEM_NOT_CONVERGED));
      } else {
        m->beta = res;
        member_cycle(*m);
        m->phase = GroupMember::ITER;
      }
    }
  }
  return 0;
}

} // namespace

extern "C" {

int stfem_group_create(stfem_group *out) {
  if (!out) return STFEM_ERR_ARG;
  stfem_group g = new stfem_group_ctx();
  cudaGetDevice(&g->device);
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming) != cudaSuccess) {
    delete g;
    return STFEM_ERR_CUDA;
  }
  *out = g;
  return STFEM_OK;
}

int stfem_group_add(stfem_group g, stfem_h h, int first_slab, int n_slabs, double *state, double tol, int restart,
                    int max_it, long long *member) {
  if (!g || !h || !state || !member || first_slab < 0 || n_slabs < 0 || restart < 1 || max_it < 0 ||
      !(tol >= 0.0))
    return STFEM_ERR_ARG;
  if (h->precision < 0) {
    g->err = "stfem_gmg_setup has not been called on the handle";
    return STFEM_ERR_STATE;
  }
  if (restart > MAXM) {
    g->err = "restart length above the supported maximum";
    return STFEM_ERR_ARG;
  }
  for (auto &m : g->members) {
    if (m->phase == GroupMember::DONE) continue;
    if (m->h == h) {
      g->err = "the handle is already a member of the group";
      return STFEM_ERR_ARG;
    }
    if (m->h->q != h->q || m->h->precision != h->precision) {
      g->err = "group members share the temporal degree and the precision";
      return STFEM_ERR_ARG;
    }
  }
  if (!h->grp_ev && cudaEventCreateWithFlags(&h->grp_ev, cudaEventDisableTiming) != cudaSuccess) {
    g->err = "cudaEventCreate failed";
    return STFEM_ERR_CUDA;
  }
  auto m = std::make_unique<GroupMember>();
  m->h = h;
  m->id = g->next_id++;
  m->first = first_slab;
  m->n_slabs = n_slabs;
  m->state = state;
  m->tol = tol;
  m->restart = restart;
  m->max_it = max_it;
  m->phase = n_slabs > 0 ? GroupMember::START : GroupMember::DONE;
  *member = m->id;
  g->members.push_back(std::move(m));
  return STFEM_OK;
}

int stfem_group_step(stfem_group g, int *n_active) {
  if (!g) return STFEM_ERR_ARG;
  const int rc = group_step(g);
  int n = 0;
  for (auto &m : g->members) n += m->phase != GroupMember::DONE && m->status >= 0;
  if (n_active) *n_active = n;
  return rc;
}

int stfem_group_member(stfem_group g, long long member, int *done, int *status, int *iters_host,
                       double *slab_ms_host) {
  if (!g) return STFEM_ERR_ARG;
  for (auto &m : g->members) {
    if (m->id != member) continue;
    const bool fin = m->phase == GroupMember::DONE || m->status < 0;
    if (done) *done = fin ? 1 : 0;
    if (status) *status = m->status;
    if (fin && m->status >= 0) {
      const int rc = check_dev_err(m->h);
      if (rc < 0) {
        m->status = rc;
        if (status) *status = rc;
      }
    }
    for (size_t i = 0; i < m->iters.size(); ++i) {
      if (iters_host) iters_host[i] = m->iters[i];
      if (slab_ms_host) slab_ms_host[i] = m->slab_ms[i];
    }
    return STFEM_OK;
  }
  g->err = "unknown group member";
  return STFEM_ERR_ARG;
}

int stfem_group_remove(stfem_group g, long long member) {
  if (!g) return STFEM_ERR_ARG;
  for (size_t i = 0; i < g->members.size(); ++i)
    if (g->members[i]->id == member) {
      if (cudaStreamSynchronize(g->members[i]->h->stream) != cudaSuccess) return STFEM_ERR_CUDA;
      g->members.erase(g->members.begin() + i);
      return STFEM_OK;
    }
  g->err = "unknown group member";
  return STFEM_ERR_ARG;
}

int stfem_group_stats(stfem_group g, long long *fused_launches, long long *fused_jobs) {
  if (!g) return STFEM_ERR_ARG;
  if (fused_launches) *fused_launches = g->fused_launches;
  if (fused_jobs) *fused_jobs = g->fused_jobs;
  return STFEM_OK;
}

const char *stfem_group_last_error(stfem_group g) { return g ? g->err.c_str() : ""; }

void stfem_group_destroy(stfem_group g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  for (auto &m : g->members)
    if (m->h) cudaStreamSynchronize(m->h->stream);
  cudaEventDestroy(g->ev);
  cudaStreamDestroy(g->stream);
  delete g;
}

} // extern "C"
