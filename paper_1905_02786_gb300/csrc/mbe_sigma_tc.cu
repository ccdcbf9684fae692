// Fused mixed-precision sigma vector on the 5th-generation tensor cores
// (tcgen05, sm_103a): string-pair gather of D into shared memory, the
// (kl|ij) contraction E = g' D as split-BF16x3 MMAs with an FP32 accumulator
// in tensor memory, and the scatter of E into the sigma rows, in one kernel.
//
// With c symmetric (the alpha<->beta symmetric Davidson vectors), D and E
// are symmetric in the two string indices, so the alpha half of the scatter
// is the transpose of the beta half: sigma = X + X^T with
//   X(a, b) = 1/2 sum_P sum_k <b|E+_P|k> E_P(a, k)        (beta strings)
// Each CTA owns R full rows a of X (kept in shared memory, no global
// atomics) and walks the column strings k in tiles; for a tile of
// M = 128 determinants (a, k) it
//   1. gathers D_P(a,k) = s_a c(J_a,k) + s_k c(a,J_k) for all pairs P
//      (rows J_a of c read coalesced from global memory, row a of c staged in
//      shared memory, the link rows of the tile's column strings staged as
//      int16) and splits it into bf16 hi + lo as the A operand (one
//      determinant per row, K = pairs, K-major core-matrix layout, 16-byte
//      vector stores),
//   2. one elected thread issues D_hi g'_hi + D_lo g'_hi + D_hi g'_lo as
//      tcgen05.mma (M = 128 determinants, N = kpad pairs, K = 16 per
//      instruction; g' is symmetric, so this is E^T) into an FP32
//      accumulator in TMEM and commits to an mbarrier,
//   3. every warp reads E^T back with tcgen05.ld (warp w: TMEM lanes
//      32 (w mod 4) .. + 31 = determinants, every other 8-column chunk of
//      pairs) and pushes 1/2 s E_P(a,k) into X(a, J) for the string J linked
//      to k by P (shared-memory atomics); all eight warps carry equal work.
// Precision: both operands carry ~16 significant bits after the hi/lo split,
// the dropped lo*lo term and the FP32 accumulation give sigma to ~1e-4 of
// its largest element; the Davidson iteration corrects this with FP64-grade
// sigma vectors.  Input c and output sigma are FP32 (no FP64 arithmetic on
// the per-element path: GB300's FP64 pipe is a small fraction of FP32).
#include "mbe_internal.cuh"
#include "mbe_tcgen05.cuh"
#include <cuda_bf16.h>
#include <algorithm>

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_N = 128;        // determinants per MMA tile (R rows x W cols)
constexpr int TC_M = 128;        // MMA M (= TC_N determinants); npair <= 128
using namespace tc5;

struct TcShared {
  // byte offsets into dynamic shared memory
  uint32_t d_hi, d_lo, g_hi, g_lo, c_rows, x_rows, link_k, link_a, total;
};

// row stride (int16) of the staged link rows: kpad entries (-1 beyond
// npair) rounded to an odd number of 16-byte units, so that 8-pair blocks
// are single 16-byte loads and 32 rows read the same block conflict-free
__host__ __device__ inline int link_stride(int kpad) { return 8 * ((kpad >> 3) | 1); }

__host__ __device__ inline TcShared tc_layout(int kpad, int R, int nstr, int npair, int W) {
  TcShared s;
  uint32_t o = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t r = o;
    o += (bytes + 127u) & ~127u;
    return r;
  };
  s.d_hi = take((uint32_t)TC_M * kpad * 2);
  s.d_lo = take((uint32_t)TC_M * kpad * 2);
  s.g_hi = take((uint32_t)kpad * kpad * 2);
  s.g_lo = take((uint32_t)kpad * kpad * 2);
  s.c_rows = take((uint32_t)R * (nstr + 1) * 4);
  s.x_rows = take((uint32_t)R * nstr * 4);
  s.link_k = take((uint32_t)2 * W * link_stride(kpad) * 2);
  s.link_a = take((uint32_t)R * kpad * 8);      // offsets, then signs
  s.total = o;
  return s;
}

__host__ __device__ inline uint32_t tmem_cols_for(int kpad) {
  uint32_t c = 32;
  while (c < (uint32_t)kpad) c <<= 1;
  return c;
}

// Split of g'/2 into bf16 hi + lo in the K-major core-matrix layout, once per
// tuple (the sigma kernel copies its first kpad rows into shared memory):
// gsplit[b] = {hi[128 x kpad], lo[128 x kpad]}, rows >= npair and K >= npair 0.
// The factor 1/2 of sigma = X + X^T is carried here (exact: a power of two).
__global__ void k_split_gp(const double* __restrict__ gp_all, int npair, int kpad,
                           uint8_t* __restrict__ gsplit) {
  const int b = blockIdx.y;
  const double* g = gp_all + (int64_t)b * npair * npair;
  const uint32_t slice = (uint32_t)TC_M * kpad * 2;
  uint8_t* hi = gsplit + (int64_t)b * 2 * slice;
  uint8_t* lo = hi + slice;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < TC_M * (kpad >> 3);
       it += gridDim.x * blockDim.x) {
    const int row = it / (kpad >> 3), kb = (it % (kpad >> 3)) * 8;
    __align__(16) __nv_bfloat16 h8[8], l8[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int k = kb + j;
      const double dv = (row < npair && k < npair) ? 0.5 * g[(int64_t)row * npair + k] : 0.0;
      const __nv_bfloat16 hh = __double2bfloat16(dv);
      h8[j] = hh;
      l8[j] = __double2bfloat16(dv - (double)__bfloat162float(hh));
    }
    const uint32_t off = kmajor_offset(row, kb, kpad);
    *(uint4*)(hi + off) = *(uint4*)h8;
    *(uint4*)(lo + off) = *(uint4*)l8;
  }
}

// One CTA = tuple b (blockIdx.y) x rows [a0, a0 + R) of X (blockIdx.x).  An
// MMA tile is M = 128 determinants m = r W + j <-> (a0 + r, k0 + j), r < R,
// j < W = 128 / R; the accumulator holds E^T (lane m, column P), computed
// as D^T g' (g' is symmetric) with N = kpad pair columns.  kpad (the pair
// count rounded up to 16) is a template parameter: loop trip counts, the
// operand layout and the link stride are compile-time constants.
template <int R, int KP>
__global__ void __launch_bounds__(TC_THREADS, 2)
k_sigma_tc(const int32_t* __restrict__ link, int nstr, int npair,
           const uint8_t* __restrict__ gsplit, const float* __restrict__ c, int64_t c_stride,
           const int32_t* __restrict__ active, float* __restrict__ X, int64_t x_stride,
           int32_t* __restrict__ err) {
  constexpr int W = TC_N / R;
  constexpr int kpad = KP;
  constexpr int LS = 8 * ((KP >> 3) | 1);     // link_stride(kpad)
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int a0 = blockIdx.x * R;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  const TcShared L = tc_layout(kpad, R, nstr, npair, W);
  uint8_t* sD_hi = smem + L.d_hi;
  uint8_t* sD_lo = smem + L.d_lo;
  uint8_t* sG_hi = smem + L.g_hi;
  uint8_t* sG_lo = smem + L.g_lo;
  float* sC = (float*)(smem + L.c_rows);
  float* sX = (float*)(smem + L.x_rows);
  uint16_t* sLk = (uint16_t*)(smem + L.link_k);   // [j][LS]
  int32_t* sLa = (int32_t*)(smem + L.link_a);     // [r][kpad] element offsets J nstr
  float* sLm = (float*)(sLa + R * kpad);           // [r][kpad] sign, 0 without a link
  const float* cb = c + (int64_t)b * c_stride;
  const uint32_t tcols = tmem_cols_for(kpad);

  // ---- setup: the first kpad rows of the pre-split g' into shared memory
  {
    const uint32_t slice = (uint32_t)TC_M * kpad * 2;
    const uint4* src = (const uint4*)(gsplit + (int64_t)b * 2 * slice);
    uint4* dhi = (uint4*)sG_hi;
    uint4* dlo = (uint4*)sG_lo;
    const int n16 = (int)(slice >> 4), m16 = (kpad * kpad * 2) >> 4;
    for (int i = tid; i < m16; i += TC_THREADS) {
      dhi[i] = src[i];
      dlo[i] = src[n16 + i];
    }
  }
  // rows a of c with one zero pad element each (row stride nstr + 1): the
  // column-link encoding below points missing links at the pad
  for (int it = tid; it < R * (nstr + 1); it += TC_THREADS) {
    const int r = it / (nstr + 1), k = it - r * (nstr + 1);
    const int a = a0 + r;
    sC[it] = (a < nstr && k < nstr) ? cb[a * nstr + k] : 0.f;
  }
  for (int it = tid; it < R * nstr; it += TC_THREADS) sX[it] = 0.f;
  // row links as an element offset J nstr and a sign (0 where there is no
  // link: the load then reads column k of row 0 and is multiplied away)
  for (int it = tid; it < R * kpad; it += TC_THREADS) {
    const int r = it / kpad, P = it - r * kpad;
    const int a = a0 + r;
    const int t = (a < nstr && P < npair) ? link[a * npair + P] : -1;
    sLa[it] = t < 0 ? 0 : (t >> 1) * nstr;
    sLm[it] = t < 0 ? 0.f : ((t & 1) ? -1.f : 1.f);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  constexpr uint32_t idesc = make_idesc(TC_M, kpad);
  constexpr uint32_t sbo = (uint32_t)(kpad >> 3) * 128u;
  constexpr int nkb = kpad >> 3;
  uint32_t phase = 0;
  bool ok = true;

  // gather mapping: thread -> determinant m = tid % 128 (fixed), P-blocks
  // pb = 8 (tid / 128 + 2 i)
  const int gm = tid & (TC_M - 1);
  const int gr = gm / W, gj = gm % W;            // W is a power of two
  const int ga = a0 + gr;
  const int32_t* la = sLa + gr * kpad;
  const float* lm = sLm + gr * kpad;
  const float* crow = sC + gr * (nstr + 1);
  // epilogue mapping: warp w reads TMEM lanes 32 (w mod 4) + lane = m and
  // the 8-column chunks ch = w / 4, w / 4 + 2, ... of the pair columns
  const int em = 32 * (warp & 3) + lane;
  const int er = em / W, ej = em % W;
  float* xrow = sX + er * nstr;
  const uint32_t xrow_s = smem_u32(xrow);

  // link rows of the column strings of tile kt (contiguous in link) into
  // buffer buf of sLk, one warp per row, encoded as J | negative << 15 with a
  // missing link (and every pair beyond npair or column beyond nstr) as the
  // pad index nstr, so that the gather needs no branch
  auto stage_links = [&](int kt, int buf) {
    const int nc = min(W, nstr - kt);
    uint16_t* base = sLk + buf * W * LS;
    for (int j = warp; j < W; j += TC_THREADS / 32) {
      uint16_t* dst = base + j * LS;
      const int32_t* src = link + (int64_t)(kt + j) * npair;
      int32_t v[4];
#pragma unroll
      for (int u = 0; u < 4; u++) v[u] = (j < nc && lane + 32 * u < npair) ? src[lane + 32 * u] : -1;
#pragma unroll
      for (int u = 0; u < 4; u++)
        if (lane + 32 * u < kpad)
          dst[lane + 32 * u] =
              (uint16_t)(v[u] < 0 ? nstr : ((v[u] >> 1) | ((v[u] & 1) << 15)));
    }
  };
  stage_links(0, 0);
  __syncthreads();
  int cur = 0;
  for (int k0 = 0; k0 < nstr && ok; k0 += W, cur ^= 1) {
    const uint16_t* lkg = sLk + cur * W * LS + gj * LS;
    // ---- gather D^T rows (determinant (a0 + r, k0 + j))
    {
      const int k = k0 + gj;
      const bool col_ok = ga < nstr && k < nstr;
      // column k of c (row stride nstr); column 0 stands in for an invalid
      // determinant so that the loads below need no branch
      const float* ccol = cb + (col_ok ? k : 0);
      // nkb is even (kpad is a multiple of 16): nkb / 2 blocks of 8 pairs per
      // thread.  Software pipelined: the eight row-link loads (from L2) of
      // block jb + 1 are issued before block jb is combined and stored, so
      // that their latency overlaps the arithmetic (a missing link has
      // offset 0 and sign 0; D rows of determinants beyond nstr are never
      // scattered, so they need no masking, and their loads stay in bounds
      // through ccol)
      float xa[8];
      {
        const int pb = (tid >> 7) * 8;
        const int4 a0v = *reinterpret_cast<const int4*>(la + pb);
        const int4 a1v = *reinterpret_cast<const int4*>(la + pb + 4);
        const int ta[8] = {a0v.x, a0v.y, a0v.z, a0v.w, a1v.x, a1v.y, a1v.z, a1v.w};
#pragma unroll
        for (int q = 0; q < 8; q++) xa[q] = ccol[ta[q]];
      }
#pragma unroll
      for (int jb = 0; jb < nkb / 2; jb++) {
        const int kb = (tid >> 7) + 2 * jb;
        const int pb = kb * 8;
        float xn[8];
        if (jb + 1 < nkb / 2) {
          const int4 a0v = *reinterpret_cast<const int4*>(la + pb + 16);
          const int4 a1v = *reinterpret_cast<const int4*>(la + pb + 20);
          const int tn[8] = {a0v.x, a0v.y, a0v.z, a0v.w, a1v.x, a1v.y, a1v.z, a1v.w};
#pragma unroll
          for (int q = 0; q < 8; q++) xn[q] = ccol[tn[q]];
        }
        // 8 pairs at once: one 16-byte load of the column link, two of the
        // row-link signs
        const int4 kv = *reinterpret_cast<const int4*>(lkg + pb);
        const uint32_t kw[4] = {(uint32_t)kv.x, (uint32_t)kv.y, (uint32_t)kv.z, (uint32_t)kv.w};
        const float4 m0v = *reinterpret_cast<const float4*>(lm + pb);
        const float4 m1v = *reinterpret_cast<const float4*>(lm + pb + 4);
        const float sa[8] = {m0v.x, m0v.y, m0v.z, m0v.w, m1v.x, m1v.y, m1v.z, m1v.w};
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const uint32_t e = (kw[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
          const float x = crow[e & 0x7FFFu];          // 0 at the pad
          v[q] = fmaf(sa[q], xa[q], __int_as_float(__float_as_int(x) ^ ((e & 0x8000u) << 16)));
        }
        if (jb + 1 < nkb / 2) {
#pragma unroll
          for (int q = 0; q < 8; q++) xa[q] = xn[q];
        }
        // split into bf16 hi + lo, two values per conversion
        uint4 hv, lv;
        uint32_t* hw = &hv.x;
        uint32_t* lw = &lv.x;
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
          const float2 hf = __bfloat1622float2(h2);
          const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
          hw[q] = *reinterpret_cast<const uint32_t*>(&h2);
          lw[q] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        const uint32_t off = kmajor_offset(gm, pb, kpad);
        *(uint4*)(sD_hi + off) = hv;
        *(uint4*)(sD_lo + off) = lv;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- MMA: E^T = D_hi g'_hi + D_lo g'_hi + D_hi g'_lo
    if (tid == 0) {
      const uint32_t dhi = smem_u32(sD_hi), dlo = smem_u32(sD_lo);
      const uint32_t ghi = smem_u32(sG_hi), glo = smem_u32(sG_lo);
      uint32_t acc = 0;
      for (int ks = 0; ks < (kpad >> 4); ks++) {
        const uint32_t koff = (uint32_t)ks * 256u;
        mma_bf16(tmem, make_desc(dhi + koff, 128, sbo), make_desc(ghi + koff, 128, sbo), idesc, acc);
        acc = 1;
        mma_bf16(tmem, make_desc(dlo + koff, 128, sbo), make_desc(ghi + koff, 128, sbo), idesc, 1);
        mma_bf16(tmem, make_desc(dhi + koff, 128, sbo), make_desc(glo + koff, 128, sbo), idesc, 1);
      }
      mma_commit(&mbar);
    }
    // the next tile's link rows load while the MMA runs (the other buffer is
    // free: its last reader, the previous epilogue, ended at a barrier)
    if (k0 + W < nstr) stage_links(k0 + W, cur ^ 1);
    const int timed_out = mbar_wait(&mbar, phase) ? 0 : 1;
    if (__syncthreads_or(timed_out)) {
      ok = false;
      if (tid == 0) atomicExch(err, MBE_ECUDA);
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: E^T from TMEM (g' carries the 1/2), push s E into the X row of m
    // (rows a >= nstr accumulate zeros into an unused X row; columns beyond
    // nstr carry the pad index and are skipped)
    if (ok) {
      const uint16_t* lke = sLk + cur * W * LS + ej * LS;
      const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
      // chunks ch = warp / 4 + 2 j, j < nkb / 2, two TMEM loads per wait
#pragma unroll
      for (int j = 0; j < nkb / 2; j += 2) {
        const int ch0 = (warp >> 2) + 2 * j;
        const bool two = j + 1 < nkb / 2;
        float e[16];
        if (two)
          tmem_ld8x2(tl + (uint32_t)(ch0 * 8), tl + (uint32_t)(ch0 * 8 + 16), e);
        else
          tmem_ld8(tl + (uint32_t)(ch0 * 8), e);
#pragma unroll
        for (int h = 0; h < 2; h++) {
          if (h == 1 && !two) break;
          const int ch = ch0 + 2 * h;
          const int4 kv = *reinterpret_cast<const int4*>(lke + ch * 8);
          const uint32_t kw[4] = {(uint32_t)kv.x, (uint32_t)kv.y, (uint32_t)kv.z, (uint32_t)kv.w};
#pragma unroll
          for (int q = 0; q < 8; q++) {
            const uint32_t t = (kw[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
            const uint32_t J = t & 0x7FFFu;
            const float val = __int_as_float(__float_as_int(e[8 * h + q]) ^ ((t & 0x8000u) << 16));
            // predicated shared-memory reduction (no branch): skipped at the pad
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, %3;\n\t"
                "@p red.shared.add.f32 [%0], %1;\n\t}\n" ::"r"(xrow_s + 4u * J),
                "f"(val), "r"(J), "r"((uint32_t)nstr)
                : "memory");
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // ---- write the X rows
  for (int it = tid; it < R * nstr; it += TC_THREADS) {
    const int r = it / nstr, k = it - r * nstr;
    const int a = a0 + r;
    if (a < nstr) X[(int64_t)b * x_stride + a * nstr + k] = sX[it];
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// sigma(a,b) = X(a,b) + X(b,a) + shift (S^2 c)(a,b), FP32 output
__global__ void k_sigma_tc_finish(const float* __restrict__ X, int64_t x_stride,
                                  const int32_t* __restrict__ link, const uint32_t* __restrict__ masks,
                                  int nstr, int n, int nsig, const float* __restrict__ c,
                                  int64_t c_stride, float shift, const int32_t* __restrict__ active,
                                  float* __restrict__ out, int64_t out_stride) {
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  // 32 x 32 tile with its transpose staged in shared memory
  __shared__ float tT[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const float* Xb = X + (int64_t)b * x_stride;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int row = bx + i, col = by + threadIdx.x;     // element (bx+i, by+tx) of X
    tT[threadIdx.x][i] = (row < nstr && col < nstr) ? Xb[(int64_t)row * nstr + col] : 0.f;
  }
  __syncthreads();
  const int npair = n * (n + 1) / 2;
  const float* cb = c + (int64_t)b * c_stride;
  float* ob = out + (int64_t)b * out_stride;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int ia = by + i, ib = bx + threadIdx.x;       // output (ia, ib): X(ia,ib) + X(ib,ia)
    if (ia >= nstr || ib >= nstr) continue;
    const int64_t idx = (int64_t)ia * nstr + ib;
    float v = Xb[idx] + tT[i][threadIdx.x];
    if (shift != 0.f) {
      // (S^2 c)(a, b) = (S^2 c)(b, a) for symmetric c: evaluate it for
      // (min, max) so that both elements get bitwise the same value
      const int lo = min(ia, ib), hi = max(ia, ib);
      const int32_t* la = link + (int64_t)lo * npair;
      const int32_t* lb = link + (int64_t)hi * npair;
      const uint32_t ma = masks[lo], mb = masks[hi];
      float s2 = (float)(nsig - __popc(ma & mb)) * cb[(int64_t)lo * nstr + hi];
      // pairs {p, q}: q open in the alpha string, p open in the beta string
      uint32_t oa = ma & ~mb;
      const uint32_t obm = mb & ~ma;
      while (oa) {
        const int q = __ffs(oa) - 1;
        oa &= oa - 1;
        uint32_t ob2 = obm;
        while (ob2) {
          const int p = __ffs(ob2) - 1;
          ob2 &= ob2 - 1;
          const int P = p > q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
          const int32_t ta = la[P], tb = lb[P];
          const float x = cb[(int64_t)(ta >> 1) * nstr + (tb >> 1)];
          s2 -= ((ta ^ tb) & 1) ? -x : x;
        }
      }
      v += shift * s2;
    }
    ob[idx] = v;
  }
}

// rows of X per CTA: a tile of 128 determinants spans W = 128 / R column
// strings, so more rows mean fewer column-link rows staged per tile
inline int tc_rows(int nstr) { return nstr <= 1024 ? 4 : (nstr <= 2048 ? 2 : 1); }

// one instantiation per (rows per CTA, padded pair count)
template <int R, int KP>
void launch_tc_kp(int device, dim3 grid, uint32_t smem, cudaStream_t st, const int32_t* link,
                  int nstr, int npair, const uint8_t* gsplit, const float* c, int64_t c_stride,
                  const int32_t* active, float* X, int64_t x_stride, int32_t* err) {
  static bool attr_done[MBE_MAX_DEVICES] = {false};
  once_per_device(attr_done, device, [] {
    CU_CHECK(cudaFuncSetAttribute(k_sigma_tc<R, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  227 * 1024 - 1024));
  });
  k_sigma_tc<R, KP><<<grid, TC_THREADS, smem, st>>>(link, nstr, npair, gsplit, c, c_stride,
                                                    active, X, x_stride, err);
}

template <int R>
void launch_tc_r(int device, int kpad, dim3 grid, uint32_t smem, cudaStream_t st,
                 const int32_t* link, int nstr, int npair, const uint8_t* gsplit, const float* c,
                 int64_t c_stride, const int32_t* active, float* X, int64_t x_stride,
                 int32_t* err) {
  switch (kpad) {
#define MBE_TC_CASE(KP)                                                                    \
  case KP:                                                                                 \
    launch_tc_kp<R, KP>(device, grid, smem, st, link, nstr, npair, gsplit, c, c_stride,   \
                        active, X, x_stride, err);                                         \
    break;
    MBE_TC_CASE(16)
    MBE_TC_CASE(32)
    MBE_TC_CASE(48)
    MBE_TC_CASE(64)
    MBE_TC_CASE(80)
    MBE_TC_CASE(96)
    MBE_TC_CASE(112)
    MBE_TC_CASE(128)
#undef MBE_TC_CASE
    default:
      throw MbeError{MBE_EINVAL, "unsupported pair padding for the tensor-core sigma"};
  }
}

void launch_tc(int device, int R, int kpad, dim3 grid, uint32_t smem, cudaStream_t st,
               const int32_t* link, int nstr, int npair, const uint8_t* gsplit, const float* c,
               int64_t c_stride, const int32_t* active, float* X, int64_t x_stride, int32_t* err) {
  if (R == 4)
    launch_tc_r<4>(device, kpad, grid, smem, st, link, nstr, npair, gsplit, c, c_stride, active,
                   X, x_stride, err);
  else if (R == 2)
    launch_tc_r<2>(device, kpad, grid, smem, st, link, nstr, npair, gsplit, c, c_stride, active,
                   X, x_stride, err);
  else
    launch_tc_r<1>(device, kpad, grid, smem, st, link, nstr, npair, gsplit, c, c_stride, active,
                   X, x_stride, err);
}

}  // namespace

bool sigma_tc_supported(int n, int nstr) {
  const int npair = n * (n + 1) / 2;
  if (npair > TC_M) return false;
  const int kpad = ((npair + 15) / 16) * 16;
  const int R = tc_rows(nstr);
  TcShared L = tc_layout(kpad, R, nstr, npair, TC_N / R);
  return L.total + 2048 <= 227 * 1024;
}

void sigma_tc(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w, const float* c, int64_t c_stride,
              float* out, int64_t out_stride, const int32_t* active, double spin_shift) {
  const int npair = bp.npair, nstr = bp.nstr;
  const int kpad = ((npair + 15) / 16) * 16;
  const int R = tc_rows(nstr);
  const TcShared L = tc_layout(kpad, R, nstr, npair, TC_N / R);
  if (L.total + 2048 > 227 * 1024 || npair > TC_M)
    throw MbeError{MBE_EINVAL, "active space too large for the tensor-core sigma"};
  const int64_t N = bp.ndet;
  if (w.Xf.n < (size_t)bp.B * N) w.Xf.reset(&ctx->pool, (size_t)bp.B * N);
  if (!w.err.ptr) w.err.reset(&ctx->pool, 1);
  // g' split once per batch (it is constant over the Davidson iteration)
  const size_t gbytes = (size_t)bp.B * 2 * TC_M * kpad * 2;
  if (bp.gsplit.n != gbytes) {
    bp.gsplit.reset(&ctx->pool, gbytes);
    k_split_gp<<<dim3(8, bp.B), 256, 0, ctx->stream>>>(bp.gp.ptr, npair, kpad, bp.gsplit.ptr);
    CU_LAUNCH_CHECK();
  }
  CU_CHECK(cudaMemsetAsync(w.err.ptr, 0, sizeof(int32_t), ctx->stream));
  dim3 grid((unsigned)((nstr + R - 1) / R), bp.B);
  cudaEvent_t ev;
  ctx->dom_timer.begin(ctx->stream, ctx->opt.timing != 0, &ev);
  launch_tc(ctx->device, R, kpad, grid, L.total, ctx->stream, bp.tab->link.ptr, nstr, npair,
            bp.gsplit.ptr, c, c_stride, active, w.Xf.ptr, N, w.err.ptr);
  CU_LAUNCH_CHECK();
  ctx->dom_timer.end(ctx->stream, ev);
  ctx->stats.dom_launches += 1;
  dim3 g2((unsigned)((nstr + 31) / 32), (unsigned)((nstr + 31) / 32), bp.B);
  k_sigma_tc_finish<<<g2, dim3(32, 8), 0, ctx->stream>>>(w.Xf.ptr, N, bp.tab->link.ptr,
                                                         bp.tab->masks.ptr, nstr, bp.n, bp.nsig, c,
                                                         c_stride, (float)spin_shift, active, out,
                                                         out_stride);
  CU_LAUNCH_CHECK();
}

int32_t sigma_tc_error(mbe_ctx* ctx, SigmaWork& w) {
  if (!w.err.ptr) return 0;
  int32_t e = 0;
  CU_CHECK(cudaMemcpyAsync(&e, w.err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CU_CHECK(cudaStreamSynchronize(ctx->stream));
  return e;
}
