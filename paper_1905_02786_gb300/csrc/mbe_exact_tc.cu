// FP64-grade sigma vector for the exact points of the mixed-precision
// Davidson iteration, fused like the tensor-core sigma: gather, contraction
// and scatter in one kernel, with no D or E intermediate in HBM.  Requires
// c = c^T with FP32 values and |c_i| <= 1 (normalised exact-point vectors).
//
// The exact point vector c is FP32 (its values are taken as exact), so
//   D_P(a,k) = s_a c(J_a, k) + s_k c(a, J_k)
// is the exact sum of two FP32 numbers.  Per determinant m = (a, k) of a
// tile, e_m bounds |d_1| + |d_2| over all pairs P (|.| < 2^e_m): from the
// largest |c| of row k and of row a (|d_1| <= max_j |c(j, k)|, |d_2| <=
// max_j |c(a, j)|, c = c^T; k_rowmax), and
//   F_P(m) = round(d_1 2^(39 - e_m)) + round(d_2 2^(39 - e_m))   (|F| <= 2^39)
// is cut into five balanced 8-bit digits, exact in bf16; g' is cut the same
// way per row with exponent e_P (once per batch, k_slice_gp_exact).  Every
// digit product is an integer below 2^14, and each group s = i + j (i, j
// slice indices, s <= 5) of at most five such products summed over K <= 80
// stays below 2^24, so its FP32 accumulator in tensor memory is exact
// (error-free slicing: Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 95
// (2012)).  The six group accumulators (6 x kpad <= 480 TMEM columns) give
// the exact integer I = sum_s acc_s 2^(8 (5 - s)) with E_P(m) =
// I 2^(e_P + e_m - 54).  The scatter X(a, J) += 1/2 s E is accumulated in
// 64-bit fixed point in shared memory: units 2^Z with Z = max_P e_P + 2 - 48
// (|c| <= 1 gives e_m <= 2, so |X| < 2^60 units and each contribution is I
// shifted right by at least 7 bits, rounded).  The rows of X are written in
// FP64; sigma = X + X^T + shift S^2 c follows in k_finish_sym_fp64.  Each
// term carries an error of at most 2^-38 (2^(e_m - 40)) of the largest |g'|.
//
// Layout of a tile, as in the tensor-core sigma: M = 128 determinants
// (R rows a of X per CTA, W = 128 / R column strings k), N = kpad pairs,
// A = D digits (K-major), B = g' digits (K-major), accumulator = E^T.
#include "mbe_internal.cuh"
#include "mbe_tcgen05.cuh"
#include <cuda_bf16.h>
#include <algorithm>

namespace {

using namespace tc5;

constexpr int EX_THREADS = 640;
constexpr int EX_M = 128;
constexpr int EX_SLICES = 5;
constexpr int EX_GROUPS = 6;
constexpr int EX_MAXK = 80;            // 6 groups x kpad columns <= 512
constexpr uint32_t EX_TMEM_COLS = 512;

__host__ __device__ inline int ex_link_stride(int kpad) { return 8 * ((kpad >> 3) | 1); }

// frexp exponent of an FP64 value (|x| < 2^e); -1022 for zero
__device__ __forceinline__ int exp_f64(double x) {
  const int be = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return be == 0 ? -1022 : be - 1022;
}

// frexp exponent of an FP32 value; -1000 for zero (subnormals count as zero)
__device__ __forceinline__ int exp_f32(float x) {
  const int be = (int)((__float_as_uint(x) >> 23) & 0xFF);
  return be == 0 ? -1000 : be - 126;
}

// round(x 2^(39 - e)) for |x| < 2^e, from the FP32 bit pattern (integer ops)
__device__ __forceinline__ long long fixed39_f32(float x, int e) {
  const uint32_t bits = __float_as_uint(x);
  const int be = (int)((bits >> 23) & 0xFF);
  if (be == 0) return 0;
  const long long M = (long long)((bits & 0x7FFFFFu) | 0x800000u);
  const int sh = be - 150 + 39 - e;            // x = M 2^(be - 150)
  long long F = 0;
  if (sh >= 0) F = M << sh;
  else if (sh > -40) F = (M + (1LL << (-sh - 1))) >> (-sh);
  return (bits >> 31) ? -F : F;
}

// round(x 2^(39 - e)) for an FP64 x, |x| < 2^e (integer ops)
__device__ __forceinline__ long long fixed39_f64(double x, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  if (be == 0) return 0;
  const long long M = (long long)((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const int sh = be - 1075 + 39 - e;
  long long F = 0;
  if (sh >= 0) F = M << sh;
  else if (sh > -60) F = (M + (1LL << (-sh - 1))) >> (-sh);
  return (bits >> 63) ? -F : F;
}

// the five balanced base-256 digits of F (|F| <= 2^39), most significant first
__device__ __forceinline__ void digits5(long long F, __nv_bfloat16* s) {
#pragma unroll
  for (int i = EX_SLICES - 1; i >= 1; i--) {
    const int d = (int)(signed char)(F & 0xFF);
    s[i] = __int2bfloat16_rn(d);
    F = (F - d) >> 8;
  }
  s[0] = __int2bfloat16_rn((int)F);
}

// g' of every tuple of the batch cut into digit planes: out[b] = 5 planes of
// kpad x kpad bf16 (K-major core-matrix layout), ge[b][P] = row exponents
__global__ void k_slice_gp_exact(const double* __restrict__ gp_all, int npair, int kpad,
                                 uint8_t* __restrict__ out, int32_t* __restrict__ ge) {
  const int b = blockIdx.y;
  const double* g = gp_all + (int64_t)b * npair * npair;
  const uint32_t plane = (uint32_t)kpad * kpad * 2;
  uint8_t* o = out + (int64_t)b * EX_SLICES * plane;
  __shared__ int sE[128];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int P = warp; P < kpad; P += blockDim.x >> 5) {
    double mx = 0.0;
    if (P < npair)
      for (int Q = lane; Q < npair; Q += 32) mx = fmax(mx, fabs(g[(int64_t)P * npair + Q]));
    int e = exp_f64(mx);
    for (int off = 16; off; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
    if (lane == 0) {
      sE[P] = e;
      ge[(int64_t)b * kpad + P] = e;
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < kpad * (kpad >> 3); it += blockDim.x) {
    const int row = it / (kpad >> 3), kb = (it % (kpad >> 3)) * 8;
    __align__(16) __nv_bfloat16 sl[EX_SLICES][8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int q = kb + j;
      const double x = (row < npair && q < npair) ? g[(int64_t)row * npair + q] : 0.0;
      __nv_bfloat16 d[EX_SLICES];
      digits5(fixed39_f64(x, sE[row]), d);
#pragma unroll
      for (int i = 0; i < EX_SLICES; i++) sl[i][j] = d[i];
    }
    const uint32_t off = kmajor_offset(row, kb, kpad);
#pragma unroll
    for (int i = 0; i < EX_SLICES; i++) *(uint4*)(o + i * plane + off) = *(uint4*)sl[i];
  }
}

// rmax[b][a] = max_k |c(a, k)| (one warp per row)
__global__ void k_rowmax(const float* __restrict__ c, int64_t c_stride, int nstr,
                         const int32_t* __restrict__ active, float* __restrict__ rmax) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= nstr) return;
  const float* row = c + (int64_t)b * c_stride + (int64_t)a * nstr;
  float m = 0.f;
  for (int k = lane; k < nstr; k += 32) m = fmaxf(m, fabsf(row[k]));
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) rmax[(int64_t)b * nstr + a] = m;
}

struct ExShared {
  uint32_t g, d, c_rows, x_rows, link_k, link_a, ep, em, total;
};

__host__ __device__ inline ExShared ex_layout(int kpad, int R, int nstr) {
  const int W = EX_M / R;
  ExShared s;
  uint32_t o = 0;
  auto take = [&](uint32_t bytes) {
    const uint32_t r = o;
    o += (bytes + 127u) & ~127u;
    return r;
  };
  s.g = take((uint32_t)EX_SLICES * kpad * kpad * 2);
  s.d = take((uint32_t)EX_SLICES * EX_M * kpad * 2);
  s.c_rows = take((uint32_t)R * (nstr + 1) * 4);
  s.x_rows = take((uint32_t)R * nstr * 8);
  s.link_k = take((uint32_t)W * ex_link_stride(kpad) * 2);
  s.link_a = take((uint32_t)R * kpad * 4);
  s.ep = take((uint32_t)kpad * 4);
  s.em = take((uint32_t)EX_M * 4);
  s.total = o;
  return s;
}

template <int R>
__global__ void __launch_bounds__(EX_THREADS, 1)
k_sigma_exact(const int32_t* __restrict__ link, int nstr, int npair, int kpad,
              const uint8_t* __restrict__ gslices, const int32_t* __restrict__ ge,
              const float* __restrict__ c, int64_t c_stride, const float* __restrict__ rmax,
              const int32_t* __restrict__ active, double* __restrict__ X, int64_t x_stride,
              long long wait_limit, int32_t* __restrict__ err) {
  constexpr int W = EX_M / R;
  const int LS = ex_link_stride(kpad);
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int a0 = blockIdx.x * R;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_maxep;
  const ExShared L = ex_layout(kpad, R, nstr);
  const uint32_t gplane = (uint32_t)kpad * kpad * 2, dplane = (uint32_t)EX_M * kpad * 2;
  uint8_t* sG = smem + L.g;
  uint8_t* sD = smem + L.d;
  float* sC = (float*)(smem + L.c_rows);
  long long* sX = (long long*)(smem + L.x_rows);
  uint16_t* sLk = (uint16_t*)(smem + L.link_k);
  int32_t* sLa = (int32_t*)(smem + L.link_a);
  int* sEP = (int*)(smem + L.ep);
  int* sEm = (int*)(smem + L.em);
  const float* cb = c + (int64_t)b * c_stride;

  // ---- setup: g' digit planes, row exponents, rows a of c (zero pad), X
  {
    const uint4* src = (const uint4*)(gslices + (int64_t)b * EX_SLICES * gplane);
    uint4* dst = (uint4*)sG;
    const int n16 = (int)((EX_SLICES * gplane) >> 4);
    for (int i = tid; i < n16; i += EX_THREADS) dst[i] = src[i];
  }
  if (tid == 0) s_maxep = -1022;
  __syncthreads();
  for (int P = tid; P < kpad; P += EX_THREADS) {
    const int e = ge[(int64_t)b * kpad + P];
    sEP[P] = e;
    if (P < npair) atomicMax(&s_maxep, e);
  }
  for (int it = tid; it < R * (nstr + 1); it += EX_THREADS) {
    const int r = it / (nstr + 1), k = it - r * (nstr + 1);
    const int a = a0 + r;
    sC[it] = (a < nstr && k < nstr) ? cb[a * nstr + k] : 0.f;
  }
  for (int it = tid; it < R * nstr; it += EX_THREADS) sX[it] = 0;
  for (int it = tid; it < R * kpad; it += EX_THREADS) {
    const int r = it / kpad, P = it - r * kpad;
    const int a = a0 + r;
    const int t = (a < nstr && P < npair) ? link[a * npair + P] : -1;
    sLa[it] = t < 0 ? -1 : (((t >> 1) * nstr) << 1) | (t & 1);
  }
  if (warp == 0) tmem_alloc(&tmem_base_sh, EX_TMEM_COLS);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  const int Z = s_maxep + 2 - 48;
  const uint32_t idesc = make_idesc(EX_M, kpad);
  const uint32_t sbo = (uint32_t)(kpad >> 3) * 128u;
  const int nkb = kpad >> 3;
  uint32_t phase = 0;
  bool ok = true;

  // thread -> determinant m = tid % 128 and P-blocks tid / 128 + 5 i (gather),
  // warp -> TMEM lanes 32 (w mod 4) and 8-column chunks w / 4 + 5 i (epilogue):
  // the ten blocks and chunks of kpad = 80 in two even rounds
  // (20 warps: 28.65 ms against 29.0 with 24 on the 64 x 8e/12o batch)
  const int gm = tid & (EX_M - 1);
  const int gr = gm / W, gj = gm % W;
  const int ga = a0 + gr;
  const int32_t* la = sLa + gr * kpad;
  const float* crow = sC + gr * (nstr + 1);
  const int em_ = 32 * (warp & 3) + lane;
  const int er = em_ / W, ej = em_ % W;
  long long* xrow = sX + er * nstr;

  // the two FP32 terms of D_P(m) for the 8 pairs of block pb
  auto terms = [&](int k, bool col_ok, int pb, const uint16_t* lkg, float* d1, float* d2) {
    const int4 a0v = *reinterpret_cast<const int4*>(la + pb);
    const int4 a1v = *reinterpret_cast<const int4*>(la + pb + 4);
    const int4 kv = *reinterpret_cast<const int4*>(lkg + pb);
    const int ta[8] = {a0v.x, a0v.y, a0v.z, a0v.w, a1v.x, a1v.y, a1v.z, a1v.w};
    const uint32_t kw[4] = {(uint32_t)kv.x, (uint32_t)kv.y, (uint32_t)kv.z, (uint32_t)kv.w};
    const float* ccol = cb + (col_ok ? k : 0);   // column 0 stands in for an invalid one
    float xa[8];
#pragma unroll
    for (int q = 0; q < 8; q++) xa[q] = ccol[ta[q] >= 0 ? (ta[q] >> 1) : 0];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      d1[q] = (col_ok && ta[q] >= 0) ? ((ta[q] & 1) ? -xa[q] : xa[q]) : 0.f;
      const uint32_t e = (kw[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
      const float x = crow[e & 0x7FFFu];
      d2[q] = (e & 0x8000u) ? -x : x;
    }
  };

  for (int k0 = 0; k0 < nstr && ok; k0 += W) {
    // ---- link rows of the tile's column strings (pad-encoded, as in the
    // tensor-core sigma)
    const int nc = min(W, nstr - k0);
    for (int j = warp; j < W; j += EX_THREADS / 32) {
      uint16_t* dst = sLk + j * LS;
      const int32_t* src = link + (int64_t)(k0 + j) * npair;
      for (int P = lane; P < kpad; P += 32) {
        const int t = (j < nc && P < npair) ? src[P] : -1;
        dst[P] = (uint16_t)(t < 0 ? nstr : ((t >> 1) | ((t & 1) << 15)));
      }
    }
    __syncthreads();
    const int k = k0 + gj;
    const bool col_ok = ga < nstr && k < nstr;
    const uint16_t* lkg = sLk + gj * LS;
    // ---- digit planes of D (A operand), e_m from the row maxima of c
    {
      const int e = col_ok ? exp_f32(rmax[(int64_t)b * nstr + ga] + rmax[(int64_t)b * nstr + k])
                           : -1000;
      if (tid < EX_M) sEm[gm] = e;
      for (int kb = tid >> 7; kb < nkb; kb += EX_THREADS / EX_M) {
        float d1[8], d2[8];
        terms(k, col_ok, kb * 8, lkg, d1, d2);
        __align__(16) __nv_bfloat16 sl[EX_SLICES][8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
          __nv_bfloat16 d[EX_SLICES];
          const long long F = e > -1000 ? fixed39_f32(d1[q], e) + fixed39_f32(d2[q], e) : 0;
          digits5(F, d);
#pragma unroll
          for (int i = 0; i < EX_SLICES; i++) sl[i][q] = d[i];
        }
        const uint32_t off = kmajor_offset(gm, kb * 8, kpad);
#pragma unroll
        for (int i = 0; i < EX_SLICES; i++) *(uint4*)(sD + i * dplane + off) = *(uint4*)sl[i];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- group accumulators: acc_s = sum_{i + j = s} D_i g'_j^T (columns s kpad)
    if (tid == 0) {
      const uint32_t d0 = smem_u32(sD), g0 = smem_u32(sG);
      for (int ks = 0; ks < (kpad >> 4); ks++) {
        const uint32_t koff = (uint32_t)ks * 256u;
        for (int s = 0; s < EX_GROUPS; s++) {
          bool first = true;
          for (int i = 0; i < EX_SLICES; i++) {
            const int j = s - i;
            if (j < 0 || j >= EX_SLICES) continue;
            mma_bf16(tmem + (uint32_t)(s * kpad), make_desc(d0 + i * dplane + koff, 128, sbo),
                     make_desc(g0 + j * gplane + koff, 128, sbo), idesc,
                     (ks > 0 || !first) ? 1u : 0u);
            first = false;
          }
        }
      }
      mma_commit(&mbar);
    }
    const int timed_out = mbar_wait(&mbar, phase, wait_limit) ? 0 : 1;
    if (__syncthreads_or(timed_out)) {
      ok = false;
      if (tid == 0) {
        atomicExch(err, MBE_ETIMEOUT);
        // the issued MMAs end before the accumulators are freed
        mbar_wait(&mbar, phase, SPIN_LIMIT);
      }
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: exact integers I, then X(a, J) += 1/2 s I 2^(e_P + e_m - 54)
    // in units of 2^Z (a right shift by >= 7 bits, rounded)
    if (ok) {
      const int e_m = sEm[em_];
      const uint16_t* lke = sLk + ej * LS;
      const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll 1
      for (int ch = warp >> 2; ch < nkb; ch += EX_THREADS / EX_M) {
        long long I[8];
#pragma unroll
        for (int q = 0; q < 8; q++) I[q] = 0;
#pragma unroll
        for (int s = 0; s < EX_GROUPS; s++) {
          float v[8];
          tmem_ld8(tmem + lane_off + (uint32_t)(s * kpad + ch * 8), v);
#pragma unroll
          for (int q = 0; q < 8; q++)
            I[q] += (long long)__float2int_rn(v[q]) * (1LL << (8 * (EX_GROUPS - 1 - s)));
        }
        const int4 kv = *reinterpret_cast<const int4*>(lke + ch * 8);
        const uint32_t kw[4] = {(uint32_t)kv.x, (uint32_t)kv.y, (uint32_t)kv.z, (uint32_t)kv.w};
        if (e_m > -1000) {
#pragma unroll
          for (int q = 0; q < 8; q++) {
            const uint32_t t = (kw[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
            const uint32_t J = t & 0x7FFFu;
            if (J == (uint32_t)nstr) continue;
            const int sh = Z + 54 + 1 - (sEP[ch * 8 + q] + e_m);   // >= 7
            long long v = sh < 63 ? (I[q] + (1LL << (sh - 1))) >> sh : 0;
            if (t & 0x8000u) v = -v;
            atomicAdd((unsigned long long*)&xrow[J], (unsigned long long)v);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // ---- X rows in FP64: sX 2^Z
  const double scale = __longlong_as_double((long long)(Z + 1023) << 52);
  for (int it = tid; it < R * nstr; it += EX_THREADS) {
    const int r = it / nstr, kk = it - r * nstr;
    const int a = a0 + r;
    if (a < nstr) X[(int64_t)b * x_stride + (int64_t)a * nstr + kk] = (double)sX[it] * scale;
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, EX_TMEM_COLS);
}

}  // namespace

bool sigma_exact_supported(int npair, int nstr) {
  const int kpad = ((npair + 15) / 16) * 16;
  if (kpad > EX_MAXK) return false;
  const int R = nstr <= 2048 ? 2 : 1;
  return ex_layout(kpad, R, nstr).total + 2048 <= 227 * 1024;
}

void sigma_exact_prepare(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w) {
  const int npair = bp.npair, nstr = bp.nstr;
  const int kpad = ((npair + 15) / 16) * 16;
  const int R = nstr <= 2048 ? 2 : 1;
  const ExShared L = ex_layout(kpad, R, nstr);
  if (kpad > EX_MAXK || L.total + 2048 > 227 * 1024)
    throw MbeError{MBE_EINVAL, "active space too large for the fused exact sigma"};
  if (!w.err.ptr) {
    w.err.reset(&ctx->pool, 1);
    CU_CHECK(cudaMemsetAsync(w.err.ptr, 0, sizeof(int32_t), ctx->stream));
  }
  // g' digit planes once per batch (g' is constant over the iteration)
  const size_t gbytes = (size_t)bp.B * EX_SLICES * kpad * kpad * 2;
  if (w.gex.n != gbytes) {
    w.gex.reset(&ctx->pool, gbytes);
    w.gexp.reset(&ctx->pool, (size_t)bp.B * kpad);
    k_slice_gp_exact<<<dim3(1, bp.B), 256, 0, ctx->stream>>>(bp.gp.ptr, npair, kpad, w.gex.ptr,
                                                             w.gexp.ptr);
    CU_LAUNCH_CHECK();
  }
  if (w.rmax.n < (size_t)bp.B * nstr) w.rmax.reset(&ctx->pool, (size_t)bp.B * nstr);
  static bool attr_done[MBE_MAX_DEVICES] = {false};
  once_per_device(attr_done, ctx->device, [] {
    CU_CHECK(cudaFuncSetAttribute(k_sigma_exact<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  227 * 1024 - 1024));
    CU_CHECK(cudaFuncSetAttribute(k_sigma_exact<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  227 * 1024 - 1024));
  });
}

void sigma_exact(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w, const float* c, int64_t c_stride,
                 double* X, int64_t x_stride, const int32_t* active) {
  const int npair = bp.npair, nstr = bp.nstr;
  const int kpad = ((npair + 15) / 16) * 16;
  const int R = nstr <= 2048 ? 2 : 1;
  const ExShared L = ex_layout(kpad, R, nstr);
  // one-time set-up of the batch (allocations, g' digit planes)
  sigma_exact_prepare(ctx, bp, w);
  const dim3 grid((unsigned)((nstr + R - 1) / R), bp.B);
  cudaEvent_t ev;
  ctx->fp64_timer.begin(ctx->stream, ctx->opt.timing != 0, &ev);
  k_rowmax<<<dim3((unsigned)((nstr + 7) / 8), bp.B), 256, 0, ctx->stream>>>(c, c_stride, nstr,
                                                                          active, w.rmax.ptr);
  CU_LAUNCH_CHECK();
  if (R == 2)
    k_sigma_exact<2><<<grid, EX_THREADS, L.total, ctx->stream>>>(
        bp.tab->link.ptr, nstr, npair, kpad, w.gex.ptr, w.gexp.ptr, c, c_stride, w.rmax.ptr,
        active, X, x_stride, ctx->opt.wait_limit, w.err.ptr);
  else
    k_sigma_exact<1><<<grid, EX_THREADS, L.total, ctx->stream>>>(
        bp.tab->link.ptr, nstr, npair, kpad, w.gex.ptr, w.gexp.ptr, c, c_stride, w.rmax.ptr,
        active, X, x_stride, ctx->opt.wait_limit, w.err.ptr);
  CU_LAUNCH_CHECK();
  ctx->fp64_timer.end(ctx->stream, ev);
  ctx->stats.fp64_launches += 1;
}
