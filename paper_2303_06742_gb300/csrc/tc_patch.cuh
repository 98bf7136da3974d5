// Batched time-diagonal patch apply on the 5th-generation tensor cores
// (tcgen05, TF32 operands, FP32 accumulators in tensor memory), for nb <= 8
// right-hand sides that share the patch inverses: the local Vanka solves of
// Algorithm 4.1 with A_P^{-1} in the time-diagonal form
// y = (V (x) I) blockdiag(Z_a) (U (x) I) r.
//
// Included by stfem.cu after the bulk-copy / mbarrier helpers.
//
// Per patch and slot a the product z_a = Z_a x_a is one GEMM D = A B with
//   real slot:    A = Z_a (Cs x Cs),            B = [X | 0]            (N = 16)
//   complex slot: A = [Re Z_a | Im Z_a] (Cs x 2Cs), B = [[Xr, Xi], [-Xi, Xr]]
// so that D = [Re z | Im z] (column n < 8: right-hand side n, real part;
// n >= 8: imaginary part).  A is stored at setup in the canonical K-major
// layout without swizzle (8 x 16-byte core matrices; per K-block of 8 values
// the row groups of 8 rows, each holding its two K cores), so a contiguous
// bulk copy lands in shared memory ready for the MMA descriptors: rows padded
// to Cs8 = 8 ceil(Cs / 8), K to Cs8 (real) or 2 Cs8 (complex), with zeros.
//
// Work items: a CTA takes items (patch p, M tiles t0 .. t1-1) from a table,
// item i = blockIdx.x, blockIdx.x + gridDim.x, ...  An item is a whole patch
// (t0 = 0, t1 = its tile count) or a single 128-row M tile of one; the rows of
// D, and so of the patch result (the time mixing with V acts row by row), are
// independent of one another, so a patch's tiles may go to different CTAs.
// An item computes its rows with the same MMA sequence as a whole patch
// (K blocks in ascending order into the same accumulator), so the result does
// not depend on how patches are cut into items or spread over CTAs.
//
// Every slot of an item has its own B operand in shared memory and its own
// accumulator in tensor memory (slot a, tile t at column 16 (a ntl + t)), so
// the MMAs of all slots run back to back, and the epilogue mixes the slots
// back to the time nodes straight from tensor memory.
//
// Warp roles (320 threads): warp 0 streams A through a ring of stages
// (cp.async.bulk, mbarrier transaction counts); warp 1 owns the tensor
// memory and one lane issues the MMAs; warps 2..9 gather and transform the
// residual columns (the next item's while the MMAs of this one run), write
// B, read D back (tcgen05.ld) and mix the result back to the time nodes.
// Every wait is bounded (clock64); on a timeout the CTA sets *err and every
// role leaves at its next uniform decision point after draining its own
// copies / MMAs.

// CTAs of the tensor-core kernel resident per SM (the registers per thread
// are bounded to fit them).
#ifndef STFEM_TC_CTAS_PER_SM
#define STFEM_TC_CTAS_PER_SM 2
#endif

namespace tcp {

constexpr int THREADS = 320;
constexpr int NCONS = 256; // consumer threads (warps 2..9)
constexpr int STAGE = 16384;
constexpr int SLACK = 4096; // the last M tile of a K block reads up to 4 KB past it
constexpr int MAXSTAGES = 8;
constexpr long long WAIT = 4000000000LL;
constexpr uint32_t IDESC = (1u << 4)         // D: FP32
                           | (2u << 7)       // A: TF32
                           | (2u << 10)      // B: TF32
                           | ((16u >> 3) << 17) // N = 16
                           | ((128u >> 4) << 24); // M = 128

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46); // descriptor version 1, no swizzle, base offset 0
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
               "l"(a), "l"(b), "r"(IDESC), "r"(accum)
               : "memory");
}

__device__ __forceinline__ void commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
               " [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                 "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 2, %0;" ::"r"(NCONS) : "memory"); }

__host__ __device__ __forceinline__ int cs8(int cs) { return (cs + 7) / 8 * 8; }
// K extent of slot a (real slots first)
__host__ __device__ __forceinline__ int kext(int a, int nr, int c8) { return a < nr ? c8 : 2 * c8; }
// first K row of slot a in the slots' stacked K extents (units of Cs8)
__host__ __device__ __forceinline__ int krow(int a, int nr) { return a < nr ? a : nr + 2 * (a - nr); }
// tensor-memory columns of the accumulators: ns slots x ntile tiles x 16,
// allocated as a power of two >= 32
__host__ __device__ inline uint32_t tmem_cols(int ns, int c8max) {
  uint32_t cols = 32;
  while (cols < (uint32_t)(16 * ns * ((c8max + 127) / 128))) cols *= 2;
  return cols;
}

struct Smem {
  unsigned char *stage; // MAXSTAGES * STAGE + SLACK (nst used)
  float *B;             // per slot 16 x K_a, core layout [kb][n group][k core]; slots stacked
  float *xt;            // [slot rows (nr + 2 nc)][8][maxCs]: transformed residual
  uint64_t *full, *empty, *bfull, *afull, *aempty, *drain;
  uint32_t *tmem;
  volatile int *flag; // [0] abort, [1] consumer decision
};

__device__ __forceinline__ Smem carve(unsigned char *base, int nst, int maxCs, int nrow) {
  Smem s;
  size_t o = 0;
  s.stage = base + o;
  o += (size_t)nst * STAGE + SLACK;
  s.B = reinterpret_cast<float *>(base + o);
  o += (size_t)16 * nrow * cs8(maxCs) * sizeof(float);
  s.xt = reinterpret_cast<float *>(base + o);
  o += (size_t)nrow * 8 * maxCs * sizeof(float);
  o = (o + 7) / 8 * 8;
  s.full = reinterpret_cast<uint64_t *>(base + o);
  s.empty = s.full + MAXSTAGES;
  s.bfull = s.empty + MAXSTAGES;
  s.afull = s.bfull + 1;
  s.aempty = s.afull + 1;
  s.drain = s.aempty + 1;
  s.tmem = reinterpret_cast<uint32_t *>(s.drain + 1);
  s.flag = reinterpret_cast<volatile int *>(s.tmem + 2);
  return s;
}

__host__ __device__ inline size_t smem_bytes(int nst, int maxCs, int nrow) {
  size_t o = (size_t)nst * STAGE + SLACK + (size_t)16 * nrow * cs8(maxCs) * sizeof(float) +
             (size_t)nrow * 8 * maxCs * sizeof(float);
  o = (o + 7) / 8 * 8;
  return o + (2 * MAXSTAGES + 4) * 8 + 16;
}

} // namespace tcp

template <int Q>
__global__ void __launch_bounds__(tcp::THREADS, STFEM_TC_CTAS_PER_SM)
    k_patch_apply_tc(int nitem, const int2 *__restrict__ items, int nb, const int *__restrict__ pcs, const long long *__restrict__ pdoff,
                     const int *__restrict__ pdofs, const long long *__restrict__ ptoff,
                     const float *__restrict__ ptile, const float *__restrict__ res, long rstride,
                     float *__restrict__ y, long ystride, DiagCoef<float> dc, int maxCs, int nst, uint32_t tcols,
                     int *__restrict__ err) {
  using namespace tcp;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  const int nr = dc.nr, nc = dc.nc, ns = nr + nc, nrow = nr + 2 * nc;
  const Smem S = carve(smem_tc, nst, maxCs, nrow);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int st = 0; st < nst; ++st) {
      mbar_init(&S.full[st], 1);
      mbar_init(&S.empty[st], 1);
    }
    mbar_init(S.bfull, 1);
    mbar_init(S.afull, 1);
    mbar_init(S.aempty, 1);
    mbar_init(S.drain, 1);
    S.flag[0] = 0;
    S.flag[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(S.tmem)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *S.tmem;

  if (warp == 0) {
    // ---------------- producer: the A stages of every (patch, slot)
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (int i = blockIdx.x; i < nitem && ok; i += gridDim.x) {
        const int2 w = items[i];
        const int p = w.x, t0 = w.y & 0xffff, t1 = w.y >> 16;
        const int c8 = cs8(pcs[p]);
        // bytes of the item's rows in one K block; a whole patch's K blocks
        // are contiguous, a tile's rows are a 4 KB-aligned piece of each
        const int rb = (min(t1 * 128, c8) - t0 * 128) * 32, per = STAGE / rb;
        const bool whole = rb == c8 * 32;
        const unsigned char *slot = reinterpret_cast<const unsigned char *>(ptile + ptoff[p]);
        for (int a = 0; a < ns && ok; ++a) {
          const int nkb = kext(a, nr, c8) / 8;
          for (int kb = 0; kb < nkb; kb += per) {
            const int st = (int)(it % nst);
            if (it >= nst && !mbar_wait(&S.empty[st], (uint32_t)(((it / nst) - 1) & 1), WAIT)) {
              ok = false;
              break;
            }
            if (S.flag[0]) {
              ok = false;
              break;
            }
            const int nk = min(per, nkb - kb);
            unsigned char *dst = S.stage + (size_t)st * STAGE;
            mbar_arrive_expect_tx(&S.full[st], (uint32_t)(nk * rb));
            if (whole) {
              bulk_copy_g2s(dst, slot + (size_t)kb * c8 * 32, (uint32_t)(nk * rb), &S.full[st]);
            } else {
              for (int j = 0; j < nk; ++j)
                bulk_copy_g2s(dst + (size_t)j * rb, slot + ((size_t)(kb + j) * c8 + (size_t)t0 * 128) * 32,
                              (uint32_t)rb, &S.full[st]);
            }
            ++it;
          }
          slot += (size_t)nkb * c8 * 32;
        }
      }
      if (!ok) {
        atomicExch(err, 3);
        S.flag[0] = 1;
        for (long long k = (it > nst ? it - nst : 0); k < it; ++k)
          mbar_wait(&S.full[k % nst], (uint32_t)((k / nst) & 1), WAIT);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      long long it = 0, nph = 0;
      bool ok = true;
      const uint32_t bbase = smem_addr(S.B);
      for (int i = blockIdx.x; i < nitem && ok; i += gridDim.x, ++nph) {
        const int2 w = items[i];
        const int p = w.x, t0 = w.y & 0xffff, t1 = w.y >> 16;
        const int c8 = cs8(pcs[p]), ntl = t1 - t0;
        const int rb = (min(t1 * 128, c8) - t0 * 128) * 32, per = STAGE / rb;
        // the item's B operands written; D free (the previous item's read back)
        if (!mbar_wait(S.bfull, (uint32_t)(nph & 1), WAIT) ||
            (nph > 0 && !mbar_wait(S.aempty, (uint32_t)((nph - 1) & 1), WAIT)) || S.flag[0]) {
          ok = false;
          break;
        }
        fence_after();
        for (int a = 0; a < ns && ok; ++a) {
          const int nkb = kext(a, nr, c8) / 8;
          const uint32_t bslot = bbase + (uint32_t)(16 * c8 * krow(a, nr)) * 4u;
          const uint32_t dslot = tbase + (uint32_t)(a * ntl * 16);
          for (int kb = 0; kb < nkb; kb += per) {
            const int st = (int)(it % nst);
            if (!mbar_wait(&S.full[st], (uint32_t)((it / nst) & 1), WAIT)) {
              ok = false;
              break;
            }
            fence_after();
            const uint32_t sbase = smem_addr(S.stage + (size_t)st * STAGE);
            const int nk = min(per, nkb - kb);
            for (int j = 0; j < nk; ++j) {
              const uint64_t bd = sdesc(bslot + (uint32_t)(kb + j) * 512u, 128u, 256u);
              for (int mt = 0; mt < ntl; ++mt) {
                const uint64_t ad = sdesc(sbase + (uint32_t)(j * rb + mt * 4096), 128u, 256u);
                mma_tf32(dslot + (uint32_t)(mt * 16), ad, bd, (kb + j) > 0 ? 1u : 0u);
              }
            }
            commit(&S.empty[st]); // stage free once these MMAs have read it
            ++it;
          }
        }
        if (!ok) break;
        commit(S.afull); // every slot's D of the item complete
      }
      if (!ok) {
        atomicExch(err, 4);
        S.flag[0] = 1;
      }
      // every MMA issued has completed before tensor memory is released
      commit(S.drain);
      mbar_wait(S.drain, 0u, WAIT);
    }
  } else {
    // ---------------- consumers (threads 64 .. 319)
    const int tid = threadIdx.x - 64;
    const int cw = tid >> 5;          // consumer warp 0..7
    const int quarter = warp & 3;     // tensor-memory lanes 32 quarter .. +31
    const int group = cw >> 2;        // tiles mt = group, group + 2, ...
    // gather the nb residual columns of patch p and transform them to the
    // slots: xt[row][c][m], row = real slot a, or 2 rows (re, im) per complex slot.
    // A thread takes one patch row m: its Q slab indices are loaded once for
    // all columns, and the 8 Q residual values behind them are all requested
    // before the first is used.
    auto gather = [&](int p) {
      const int Cs = pcs[p];
      const long long doff = pdoff[p];
      for (int m = tid; m < Cs; m += NCONS) {
        int g[Q];
#pragma unroll
        for (int b = 0; b < Q; ++b) g[b] = pdofs[doff + b * Cs + m];
        float r[8][Q];
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
          for (int b = 0; b < Q; ++b) r[c][b] = c < nb ? res[(long)c * rstride + g[b]] : 0.f;
        for (int a = 0; a < ns; ++a) {
          const bool cplx = a >= nr;
          const int row = cplx ? nr + 2 * (a - nr) : a;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int b = 0; b < Q; ++b) {
              re += dc.U[(a * Q + b) * 2] * r[c][b];
              im += dc.U[(a * Q + b) * 2 + 1] * r[c][b];
            }
            S.xt[((size_t)row * 8 + c) * maxCs + m] = re;
            if (cplx) S.xt[((size_t)(row + 1) * 8 + c) * maxCs + m] = im;
          }
        }
      }
    };
    // B operand of slot a from xt (see the layout above), at its place in the
    // stacked slots
    auto write_b = [&](int a, int Cs, int c8) {
      const int K = kext(a, nr, c8);
      const bool cplx = a >= nr;
      const int row = krow(a, nr);
      float *Bs = S.B + (size_t)16 * c8 * row;
      // a thread writes one 16-byte core row: k0 .. k0 + 3 of column n
      for (int idx = tid; idx < 4 * K; idx += NCONS) {
        const int k0 = (idx >> 4) * 4, n = idx & 15;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = k0 + e;
          v[e] = 0.f;
          if (!cplx) {
            if (n < 8 && k < Cs) v[e] = S.xt[((size_t)row * 8 + n) * maxCs + k];
          } else {
            const int kk = k < c8 ? k : k - c8;
            if (kk < Cs) {
              const float xr = S.xt[((size_t)row * 8 + (n & 7)) * maxCs + kk];
              const float xi = S.xt[((size_t)(row + 1) * 8 + (n & 7)) * maxCs + kk];
              v[e] = k < c8 ? (n < 8 ? xr : xi) : (n < 8 ? -xi : xr);
            }
          }
        }
        const int kb = k0 >> 3, kc = (k0 >> 2) & 1, ng = n >> 3, rr = n & 7;
        *reinterpret_cast<float4 *>(&Bs[(size_t)kb * 128 + (ng * 2 + kc) * 32 + rr * 4]) =
            make_float4(v[0], v[1], v[2], v[3]);
      }
    };
    // The next item's patch is gathered while the MMAs of this one run; the
    // epilogue mixes every slot's D straight back to the time nodes:
    // y_b = sum over real slots V_ba z_a + sum over complex slots 2 Re(V_ba z_a).
    long long nph = 0;
    if (blockIdx.x < nitem) gather(items[blockIdx.x].x);
    for (int i = blockIdx.x; i < nitem; i += gridDim.x, ++nph) {
      cons_sync(); // xt of the item's patch complete
      if (tid == 0) S.flag[1] = S.flag[0];
      cons_sync();
      if (S.flag[1]) break;
      const int2 w = items[i];
      const int p = w.x, t0 = w.y & 0xffff, ntl = (w.y >> 16) - t0;
      const int Cs = pcs[p], c8 = cs8(Cs);
      const long long doff = pdoff[p];
      for (int a = 0; a < ns; ++a) write_b(a, Cs, c8);
      fence_async_smem();
      cons_sync();
      if (tid == 0) mbar_arrive(S.bfull);
      if (i + (int)gridDim.x < nitem) gather(items[i + gridDim.x].x);
      if (tid == 0) S.flag[1] = mbar_wait(S.afull, (uint32_t)(nph & 1), WAIT) ? 0 : 1;
      cons_sync();
      if (S.flag[1]) {
        if (tid == 0) {
          atomicExch(err, 5);
          S.flag[0] = 1;
        }
        break;
      }
      fence_after();
      for (int mt = group; mt < ntl; mt += 2) {
        float o[8][Q];
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
          for (int b = 0; b < Q; ++b) o[c][b] = 0.f;
        for (int a = 0; a < ns; ++a) {
          float v[16];
          __syncwarp();
          ld16(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((a * ntl + mt) * 16), v);
          if (a < nr) {
#pragma unroll
            for (int b = 0; b < Q; ++b) {
              const float vr = dc.V[(b * ns + a) * 2];
#pragma unroll
              for (int c = 0; c < 8; ++c) o[c][b] += vr * v[c];
            }
          } else {
#pragma unroll
            for (int b = 0; b < Q; ++b) {
              const float vr = dc.V[(b * ns + a) * 2], vi = dc.V[(b * ns + a) * 2 + 1];
#pragma unroll
              for (int c = 0; c < 8; ++c) o[c][b] += 2.f * (vr * v[c] - vi * v[8 + c]);
            }
          }
        }
        const int m = (t0 + mt) * 128 + quarter * 32 + lane;
        if (m < Cs)
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (c < nb)
#pragma unroll
              for (int b = 0; b < Q; ++b) y[(long)c * ystride + doff + b * Cs + m] = o[c][b];
      }
      fence_before();
      cons_sync();
      if (tid == 0) mbar_arrive(S.aempty);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(tcols) : "memory");
  }
}
