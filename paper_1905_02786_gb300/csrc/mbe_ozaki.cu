// FP64-grade (kl|ij) contraction E = g' D on the tcgen05 tensor cores by
// error-free slicing (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 95
// (2012)): every row of g' and every column of D is scaled by a power of two
// and cut into five signed 8-bit slices (|s_i| <= 128, exact in bf16),
//   x = 2^e (s_0 2^-7 + s_1 2^-15 + s_2 2^-23 + s_3 2^-31 + s_4 2^-39)
//       + O(2^(e-40)),
// so each slice product is an integer below 2^14 and a sum over K <= 120 of
// at most five such products per group stays below 2^24: the FP32
// accumulator of every group s = i + j (i, j = slice indices, s <= 5) is
// exact.  The six group accumulators live side by side in tensor memory; the
// epilogue combines them in FP64 with their weights 2^(e_P + e_n - 14 - 8 s).
// The result carries ~40 significant bits of every operand (error ~1e-12
// relative to the row/column maxima); the Rayleigh quotients and residuals
// of the mixed-precision Davidson iteration are evaluated with it.
//
// Layout: D[b][P][k] (FP64, k = determinant), g'[b][P][Q]; E[b][P][k] is
// written as a float pair (hi, lo) with E = hi + lo (~48 bits) in the slot
// of an FP64 element.
// One CTA: one tuple, a strided set of 64-determinant column tiles; the g'
// slices stay in shared memory for all its tiles.
#include "mbe_internal.cuh"
#include "mbe_tcgen05.cuh"
#include <cuda_bf16.h>
#include <algorithm>

namespace {

constexpr int OZ_THREADS = 256;
constexpr int OZ_M = 128;        // pair rows (npair <= 120, zero padded)
constexpr int OZ_N = 64;         // determinants per tile
constexpr int OZ_SLICES = 5;
constexpr int OZ_GROUPS = 6;     // s = i + j = 0..5
constexpr uint32_t OZ_TMEM_COLS = 512;
using namespace tc5;

// GB300 runs FP64 arithmetic at a small fraction of its integer rate, so
// scaling and slicing work on the FP64 bit pattern with integer operations.

// e with |x| < 2^e (frexp exponent) from the biased exponent field; zero and
// subnormals give -1022 (they slice to 0 against any column scale)
__device__ __forceinline__ int exp_bits(double x) {
  const int be = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return be == 0 ? -1022 : be - 1022;
}

// the five balanced base-256 digits of F = rint(x 2^(39 - e)) (|x| < 2^e):
// F = s_0 2^32 + s_1 2^24 + s_2 2^16 + s_3 2^8 + s_4, s_1..4 in [-128, 127]
__device__ __forceinline__ void slice_bits(double x, int e, __nv_bfloat16* s) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  long long F = 0;
  if (be != 0) {
    const long long M = (long long)((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const int sh = be - 1075 + 39 - e;          // x = M 2^(be - 1075)
    if (sh >= 0) F = M << sh;
    else if (sh > -60) F = (M + (1LL << (-sh - 1))) >> (-sh);
    if (bits >> 63) F = -F;
  }
#pragma unroll
  for (int i = OZ_SLICES - 1; i >= 1; i--) {
    const int d = (int)(signed char)(F & 0xFF);
    s[i] = __int2bfloat16_rn(d);
    F = (F - d) >> 8;
  }
  s[0] = __int2bfloat16_rn((int)F);
}

struct OzLayout {
  uint32_t a, b, ea, eb, total;   // a: slices of g', b: slices of the D tile
};

__host__ __device__ inline OzLayout oz_layout(int kpad) {
  OzLayout L;
  uint32_t o = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t r = o;
    o += (bytes + 127u) & ~127u;
    return r;
  };
  L.a = take((uint32_t)OZ_SLICES * OZ_M * kpad * 2);
  L.b = take((uint32_t)OZ_SLICES * OZ_N * kpad * 2);
  L.ea = take(OZ_M * 4);
  L.eb = take(OZ_N * 4);
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
k_contract_ozaki(const double* __restrict__ gp_all, int npair, int kpad,
                 const double* __restrict__ D, int64_t ndet, const int32_t* __restrict__ active,
                 const int32_t* __restrict__ bmap, double* __restrict__ E, long long wait_limit,
                 int32_t* __restrict__ err) {
  const int bl = blockIdx.y;
  const int b = bmap[bl];
  if (active && !active[b]) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  const OzLayout L = oz_layout(kpad);
  uint8_t* sA = smem + L.a;
  uint8_t* sB = smem + L.b;
  int* sEa = (int*)(smem + L.ea);
  int* sEb = (int*)(smem + L.eb);
  const uint32_t a_slice_bytes = (uint32_t)OZ_M * kpad * 2;
  const uint32_t b_slice_bytes = (uint32_t)OZ_N * kpad * 2;
  const double* g = gp_all + (int64_t)b * npair * npair;
  const double* Db = D + (int64_t)bl * npair * ndet;
  float2* E2 = reinterpret_cast<float2*>(E) + (int64_t)bl * npair * ndet;

  // ---- row exponents and slices of g'
  for (int P = warp; P < OZ_M; P += OZ_THREADS / 32) {
    double m = 0.0;
    if (P < npair)
      for (int Q = lane; Q < npair; Q += 32) m = fmax(m, fabs(g[(int64_t)P * npair + Q]));
    // (one pass over g' per CTA; the per-tile work below is integer-only)
    int em = exp_bits(m);
    for (int off = 16; off; off >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, off));
    if (lane == 0) sEa[P] = em;
  }
  __syncthreads();
  for (int it = tid; it < OZ_M * (kpad >> 3); it += OZ_THREADS) {
    const int row = it / (kpad >> 3), kb = (it % (kpad >> 3)) * 8;
    __align__(16) __nv_bfloat16 sl[OZ_SLICES][8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int k = kb + j;
      const double x = (row < npair && k < npair) ? g[(int64_t)row * npair + k] : 0.0;
      __nv_bfloat16 s4[OZ_SLICES];
      slice_bits(x, sEa[row], s4);
#pragma unroll
      for (int i = 0; i < OZ_SLICES; i++) sl[i][j] = s4[i];
    }
    const uint32_t off = kmajor_offset(row, kb, kpad);
#pragma unroll
    for (int i = 0; i < OZ_SLICES; i++) *(uint4*)(sA + i * a_slice_bytes + off) = *(uint4*)sl[i];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  const uint32_t idesc = make_idesc(OZ_M, OZ_N);
  const uint32_t sbo = (uint32_t)(kpad >> 3) * 128u;
  uint32_t phase = 0;

  const int64_t ntiles = (ndet + OZ_N - 1) / OZ_N;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t n0 = tile * OZ_N;
    // ---- column exponents of the D tile
    if (tid < OZ_N) sEb[tid] = -1022;
    __syncthreads();
    for (int it = tid; it < OZ_N * ((npair + 7) >> 3); it += OZ_THREADS) {
      const int n = it % OZ_N, pb = (it / OZ_N) * 8;
      const int64_t col = n0 + n;
      int em = -1022;
      if (col < ndet)
        for (int q = 0; q < 8 && pb + q < npair; q++)
          em = max(em, exp_bits(Db[(int64_t)(pb + q) * ndet + col]));
      if (em > -1022) atomicMax(&sEb[n], em);
    }
    __syncthreads();
    // ---- slices of the D tile (K-major: 8 consecutive pairs per 16 bytes)
    for (int it = tid; it < OZ_N * (kpad >> 3); it += OZ_THREADS) {
      const int n = it % OZ_N, pb = (it / OZ_N) * 8;
      const int64_t col = n0 + n;
      const int e = sEb[n];
      __align__(16) __nv_bfloat16 sl[OZ_SLICES][8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int P = pb + q;
        const double x = (P < npair && col < ndet) ? Db[(int64_t)P * ndet + col] : 0.0;
        __nv_bfloat16 s4[OZ_SLICES];
        slice_bits(x, e, s4);
#pragma unroll
        for (int i = 0; i < OZ_SLICES; i++) sl[i][q] = s4[i];
      }
      const uint32_t off = kmajor_offset(n, pb, kpad);
#pragma unroll
      for (int i = 0; i < OZ_SLICES; i++) *(uint4*)(sB + i * b_slice_bytes + off) = *(uint4*)sl[i];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- group accumulators acc_s (columns 64 s .. 64 s + 63)
    if (tid == 0) {
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      for (int ks = 0; ks < (kpad >> 4); ks++) {
        const uint32_t koff = (uint32_t)ks * 256u;
        for (int s = 0; s < OZ_GROUPS; s++) {
          bool first = true;
          for (int i = 0; i < OZ_SLICES; i++) {
            const int j = s - i;
            if (j < 0 || j >= OZ_SLICES) continue;
            const uint64_t da = make_desc(a0 + i * a_slice_bytes + koff, 128, sbo);
            const uint64_t db = make_desc(b0 + j * b_slice_bytes + koff, 128, sbo);
            mma_bf16(tmem + (uint32_t)(s * OZ_N), da, db, idesc, (ks > 0 || !first) ? 1u : 0u);
            first = false;
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar))
                   : "memory");
    }
    const int timed_out = mbar_wait(&mbar, phase, wait_limit) ? 0 : 1;
    if (__syncthreads_or(timed_out)) {
      if (tid == 0) {
        atomicExch(err, MBE_ETIMEOUT);
        // the issued MMAs end before the accumulators are freed
        mbar_wait(&mbar, phase, SPIN_LIMIT);
      }
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: E = 2^(e_P + e_n - 54) I with the exact integer
    // I = sum_s acc_s 2^(8 (5 - s)) (|I| < 2^62).  Every acc_s is an exact
    // FP32 integer and every acc_s 2^(8 (5 - s)) an exact FP32 value, so I is
    // summed with error-free FP32 transformations (TwoSum, largest group
    // first): I = S + Err exactly, with Err summed in FP32 (relative error
    // ~2^-48 of |I|); (hi, lo) = FastTwoSum(S, Err).  No 64-bit integer or
    // FP64 operation: those run on GB300's small FP64 pipe.
    {
      const int P = 32 * (warp & 3) + lane;
      const int c0 = 32 * (warp >> 2);
      const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
      for (int cc = 0; cc < 32; cc += 16) {
        float S[16], Er[16];
#pragma unroll
        for (int q = 0; q < 16; q++) S[q] = Er[q] = 0.f;
#pragma unroll
        for (int sgrp = 0; sgrp < OZ_GROUPS; sgrp++) {
          float v[16];
          tmem_ld16(tmem + lane_off + (uint32_t)(sgrp * OZ_N + c0 + cc), v);
          const float w = __int_as_float((127 + 8 * (OZ_GROUPS - 1 - sgrp)) << 23);   // 2^(8(5-s))
#pragma unroll
          for (int q = 0; q < 16; q++) {
            const float t = v[q] * w;                 // exact
            const float sn = S[q] + t;
            const float bb = sn - S[q];
            Er[q] += (S[q] - (sn - bb)) + (t - bb);
            S[q] = sn;
          }
        }
        if (P < npair) {
#pragma unroll
          for (int q = 0; q < 16; q++) {
            const int n = c0 + cc + q;
            const int64_t col = n0 + n;
            if (col < ndet) {
              const float hi = S[q] + Er[q];
              const float lo = Er[q] - (hi - S[q]);
              const int k = sEa[P] + sEb[n] - 14 - 8 * (OZ_GROUPS - 1);
              float2 o;
              o.x = ldexpf(hi, k);
              o.y = ldexpf(lo, k);
              E2[(int64_t)P * ndet + col] = o;
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
}

}  // namespace

bool ozaki_supported(int npair) {
  if (npair > OZ_M) return false;
  const int kpad = ((npair + 15) / 16) * 16;
  return oz_layout(kpad).total + 2048 <= 227 * 1024;
}

void contract_ozaki(mbe_ctx* ctx, const double* gp, int npair, const double* D, int64_t ndet,
                    int nb, const int32_t* active, const int32_t* bmap, double* E,
                    int32_t* err) {
  const int kpad = ((npair + 15) / 16) * 16;
  const OzLayout L = oz_layout(kpad);
  static bool attr_done[MBE_MAX_DEVICES] = {false};
  once_per_device(attr_done, ctx->device, [] {
    CU_CHECK(cudaFuncSetAttribute(k_contract_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  227 * 1024 - 1024));
  });
  int64_t ntiles = (ndet + OZ_N - 1) / OZ_N;
  // enough CTAs to fill the GPU; each CTA reuses its g' slices for its tiles
  int64_t per_tuple = std::max<int64_t>(1, std::min<int64_t>(ntiles, (2 * 152 + nb - 1) / nb));
  per_tuple = std::max<int64_t>(per_tuple, (ntiles + 31) / 32);
  dim3 grid((unsigned)std::min<int64_t>(per_tuple, ntiles), nb);
  k_contract_ozaki<<<grid, OZ_THREADS, L.total, ctx->stream>>>(gp, npair, kpad, D, ndet, active,
                                                                bmap, E, ctx->opt.wait_limit, err);
  CU_LAUNCH_CHECK();
}
