// Mixed-precision sigma vector on the 5th-generation tensor cores (tcgen05,
// sm_103a) for the alpha<->beta symmetric CI vectors c = c^T of the mixed
// Davidson iteration (FP32 in, FP32 out).
//
// Let L_P be the matrix of E_pq + E_qp (E_pp for p = q) between strings of
// one spin, <I|..|J> = the sign of the link table entry of I and pair P.
// The Hamiltonian of one CASCI is 1/2 sum_PQ g'_PQ (L_P x 1 + 1 x L_P)
// (L_Q x 1 + 1 x L_Q) with g' the pair integrals that carry the one-electron
// part (sigma_fp64 applies the same operator through D = E+ c, E = g' D and
// the scatter).  Multiplying out the alpha and beta factors splits it into a
// one-spin and a two-spin part (alpha and beta string operators commute):
//   sigma = H^a c + c H^a + Z,   H^a = 1/2 sum_PQ g'_PQ L_P L_Q,
//   Z = sum_PQ g'_PQ L_P c L_Q,
// H^a is symmetric, and Z is symmetric for symmetric c.  Here
//   W = H^a c + Z_u,   sigma = W + W^T + shift S^2 c   (bitwise symmetric)
// with Z_u the upper triangle of Z (a < J) and half its diagonal, so that
// the scatter of Z runs over half the strings
// computed by
//   k_build_haa  H^a row by row from the link table (FP64), split into bf16
//                hi/lo rows, once per batch;
//   k_split_c    c into bf16 hi/lo rows, once per call;
//   k_gemm_haa   W = H^a c, a dense N_str^3 GEMM (c^T = c gives the B
//                operand as rows of c);
//   k_sigma_ab   W += Z_u from Z/2 = sum_Q F_Q L_Q with
//                  F_Q(a, :) = sum_{P in links(a)} (g'_QP / 2) s_a(P) c(J_a(P), :)
//                for one string a.  The MMA operand "rows J_a(P) of c" is a
//                plain copy of rows (MN-major, cp.async), the other operand
//                the compacted rows P of g'/2 signed by s_a(P) (K = the
//                n_link pairs that link a, the same count for every string);
//                the product for 128 column strings lands in TMEM and the
//                scatter through the link table of the column strings adds
//                it into row a of W (columns J >= a) in shared memory;
//   k_sigma_tc_finish  sigma = W + W^T + shift S^2 c.
// Both products run as split-BF16x3 (hi*hi + lo*hi + hi*lo, FP32
// accumulation in TMEM): ~16 significant bits per operand, sigma to ~1e-4 of
// its largest element; the Davidson iteration corrects this with FP64-grade
// sigma vectors at its exact points.
#include "mbe_internal.cuh"
#include "mbe_tcgen05.cuh"
#include <cuda_bf16.h>
#include <algorithm>
#include <fstream>
#include <cstdio>

namespace {

using namespace tc5;
typedef __nv_bfloat16 bf16;

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// bf16 hi/lo of two FP32 values, packed two per word
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hw, uint32_t& lw) {
  const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h2);
  const __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hw = *reinterpret_cast<const uint32_t*>(&h2);
  lw = *reinterpret_cast<const uint32_t*>(&l2);
}

__device__ __forceinline__ void bar_sync_n(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// named barrier that also returns the OR of `pred` over its threads
__device__ __forceinline__ bool bar_red_or(int id, int n, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// ------------------------------------------------------------ c split
// c (rows of nstr FP32) -> bf16 hi rows then lo rows of ldc elements (zeros
// beyond nstr); cs_stride elements between tuples
__global__ void k_split_c(const float* __restrict__ c, int64_t c_stride, int nstr, int ldc,
                          const int32_t* __restrict__ active, bf16* __restrict__ cs,
                          int64_t cs_stride) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const float* cb = c + (int64_t)b * c_stride;
  bf16* hi = cs + (int64_t)b * cs_stride;
  bf16* lo = hi + (int64_t)nstr * ldc;
  const int chunks = ldc >> 3;
  const int64_t total = (int64_t)nstr * chunks;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(it / chunks), k0 = (int)(it - (int64_t)r * chunks) * 8;
    const float* src = cb + (int64_t)r * nstr;
    uint4 hv, lv;
    uint32_t* hw = &hv.x;
    uint32_t* lw = &lv.x;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int k = k0 + 2 * q;
      split2(k < nstr ? src[k] : 0.f, k + 1 < nstr ? src[k + 1] : 0.f, hw[q], lw[q]);
    }
    *reinterpret_cast<uint4*>(hi + (int64_t)r * ldc + k0) = hv;
    *reinterpret_cast<uint4*>(lo + (int64_t)r * ldc + k0) = lv;
  }
}

// the same from a packed symmetric vector (sym_index layout): one CTA per
// 32 x 32 tile pair (I, J), I <= J, reads tile (I, J) from the packed rows
// (coalesced) and writes the rows of both tiles, the transposed one through
// shared memory; the values are those k_split_c gives for the full vector
__global__ void k_split_c_sym(const float* __restrict__ c, int64_t c_stride, int nstr, int ldc,
                              const int32_t* __restrict__ active, bf16* __restrict__ cs,
                              int64_t cs_stride) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nt = (nstr + 31) / 32;
  int t = blockIdx.x, I = 0;
  while (t >= nt - I) {
    t -= nt - I;
    I++;
  }
  const int J = I + t;
  __shared__ float sC[32][33];
  const float* cb = c + (int64_t)b * c_stride;
  bf16* hi = cs + (int64_t)b * cs_stride;
  bf16* lo = hi + (int64_t)nstr * ldc;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  for (int i = ty; i < 32; i += ny) {
    const int r = I * 32 + i, k = J * 32 + tx;
    sC[i][tx] = (r < nstr && k < nstr) ? cb[sym_index(r, k, nstr)] : 0.f;
  }
  __syncthreads();
  // rows of tile I, columns of tile J (zeros from nstr up to ldc)
  for (int i = ty; i < 32; i += ny) {
    const int r = I * 32 + i, k = J * 32 + tx;
    if (r < nstr && k < ldc) {
      const float x = sC[i][tx];
      const bf16 h = __float2bfloat16_rn(x);
      hi[(int64_t)r * ldc + k] = h;
      lo[(int64_t)r * ldc + k] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
  }
  if (I == J) return;
  // rows of tile J, columns of tile I (all below nstr)
  for (int i = ty; i < 32; i += ny) {
    const int r = J * 32 + i, k = I * 32 + tx;
    if (r < nstr) {
      const float x = sC[tx][i];
      const bf16 h = __float2bfloat16_rn(x);
      hi[(int64_t)r * ldc + k] = h;
      lo[(int64_t)r * ldc + k] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
  }
}

// ------------------------------------------------------------ g'/2 split
// gh[b] = {hi[kp][kp], lo[kp][kp]}: bf16 split of g'/2 (zero beyond npair);
// the factor 1/2 of W = H^a c + Z/2 (exact: a power of two)
__global__ void k_prep_gh(const double* __restrict__ gp_all, int npair, int kp,
                          bf16* __restrict__ gh) {
  const int b = blockIdx.y;
  const double* g = gp_all + (int64_t)b * npair * npair;
  bf16* hi = gh + (int64_t)b * 2 * kp * kp;
  bf16* lo = hi + kp * kp;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < kp * kp; it += gridDim.x * blockDim.x) {
    const int P = it / kp, Q = it - P * kp;
    const double dv = (P < npair && Q < npair) ? 0.5 * g[(int64_t)P * npair + Q] : 0.0;
    const bf16 h = __double2bfloat16(dv);
    hi[it] = h;
    lo[it] = __double2bfloat16(dv - (double)__bfloat162float(h));
  }
}

// ------------------------------------------------------------ H^a
// Row a of H^a = 1/2 sum_PQ g'_PQ L_P L_Q: for every pair P linking a to
// a1 = J_a(P) and every pair Q linking a1 to a2, 1/2 g'_PQ s_a(P) s_a1(Q)
// goes to column a2.  One CTA per (string a, tuple); the row accumulates in
// FP64 in shared memory and is written as bf16 hi / lo rows of ldc.
constexpr int HAA_THREADS = 128;
__global__ void __launch_bounds__(HAA_THREADS)
k_build_haa(const int32_t* __restrict__ link, int nstr, int npair, const double* __restrict__ gp_all,
            int ldc, bf16* __restrict__ haa, int64_t h_stride) {
  extern __shared__ double srow[];
  __shared__ int sP[128], sJ[128];
  __shared__ double sS[128];
  __shared__ int snl;
  const int a = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  const double* g = gp_all + (int64_t)b * npair * npair;
  for (int k = tid; k < nstr; k += HAA_THREADS) srow[k] = 0.0;
  if (tid < 32) {
    int n = 0;
    for (int p0 = 0; p0 < npair; p0 += 32) {
      const int P = p0 + tid;
      const int t = P < npair ? link[(int64_t)a * npair + P] : -1;
      const unsigned m = __ballot_sync(0xffffffffu, t >= 0);
      if (t >= 0) {
        const int pos = n + __popc(m & ((1u << tid) - 1u));
        sP[pos] = P;
        sJ[pos] = t >> 1;
        sS[pos] = (t & 1) ? -0.5 : 0.5;
      }
      n += __popc(m);
    }
    if (tid == 0) snl = n;
  }
  __syncthreads();
  const int nl = snl;
  for (int w = tid; w < nl * npair; w += HAA_THREADS) {
    const int i = w / npair, Q = w - i * npair;
    const int t = link[(int64_t)sJ[i] * npair + Q];
    if (t >= 0) {
      const double v = sS[i] * g[(int64_t)sP[i] * npair + Q];
      atomicAdd(&srow[t >> 1], (t & 1) ? -v : v);
    }
  }
  __syncthreads();
  bf16* hi = haa + (int64_t)b * h_stride + (int64_t)a * ldc;
  bf16* lo = hi + (int64_t)nstr * ldc;
  for (int k = tid; k < ldc; k += HAA_THREADS) {
    const double x = k < nstr ? srow[k] : 0.0;
    const bf16 h = __double2bfloat16(x);
    hi[k] = h;
    lo[k] = __double2bfloat16(x - (double)__bfloat162float(h));
  }
}

// ------------------------------------------------------------ W = H^a c
// Tiles of 128 x 128 (rows a of H^a x rows b of c = columns b of c), K in
// blocks of 32 through a 3-stage cp.async ring loaded two blocks ahead (a
// stage is refilled once the MMAs of the block before have completed; 97 KB
// of shared memory, so two CTAs share an SM: 4 stages, one CTA per SM, were
// 0.7 % slower on the 64 x 8e/12o batch);
// both operands K-major (8 rows x 16 bytes core matrices, LBO 128, SBO 512);
// one elected thread issues the split-BF16x3 MMAs into a 128-column TMEM
// accumulator.
constexpr int GM_T = 128, GK_T = 32, G_STAGES = 3, G_AHEAD = 2, G_THREADS = 128;
constexpr uint32_t G_OPB = GM_T * GK_T * 2;          // bytes of one operand half (8 KB)
constexpr uint32_t G_STAGE = 4 * G_OPB;              // A hi, A lo, B hi, B lo
constexpr uint32_t G_SMEM = G_STAGES * G_STAGE + 1024;

__global__ void __launch_bounds__(G_THREADS)
k_gemm_haa(const bf16* __restrict__ haa, const bf16* __restrict__ cs, int64_t hs, int nstr, int ldc,
           const int32_t* __restrict__ active, float* __restrict__ W, int64_t w_stride,
           long long wait_limit, int32_t* __restrict__ err) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int ntm = (nstr + GM_T - 1) / GM_T;
  const int m0 = (blockIdx.x % ntm) * GM_T, n0 = (blockIdx.x / ntm) * GM_T;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(1024) uint8_t gsm[];
  uint8_t* sm = gsm + ((1024u - (smem_u32(gsm) & 1023u)) & 1023u);
  __shared__ uint64_t mbar[G_STAGES], mdone;
  __shared__ uint32_t tbase;
  const bf16* A = haa + (int64_t)b * hs;
  const bf16* Bm = cs + (int64_t)b * hs;
  const int64_t half = (int64_t)nstr * ldc;
  const int nk = (ldc + GK_T - 1) / GK_T;
  if (warp == 0) tmem_alloc(&tbase, 128);
  if (tid == 0) {
    for (int s = 0; s < G_STAGES; s++) mbar_init(&mbar[s], 1);
    mbar_init(&mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  const uint32_t sbase = smem_u32(sm);
  // one K block into a stage: 2 operands x 2 halves x 128 rows x 4 chunks
  auto load = [&](int kb, int s) {
    const uint32_t st = sbase + (uint32_t)s * G_STAGE;
    for (int it = tid; it < 4 * GM_T * 4; it += G_THREADS) {
      const int ch = it & 3, row = (it >> 2) & (GM_T - 1), hl = (it >> 9) & 1, op = it >> 10;
      const int gr = (op == 0 ? m0 : n0) + row;
      const int k = kb * GK_T + ch * 8;
      const bool ok = gr < nstr && k < ldc;
      const bf16* src = (op == 0 ? A : Bm) + hl * half + (ok ? (int64_t)gr * ldc + k : 0);
      const uint32_t dst = st + (uint32_t)(op * 2 + hl) * G_OPB +
                           (uint32_t)(((row >> 3) * (GK_T >> 3) + ch) * 128 + (row & 7) * 16);
      cp_async16(dst, src, ok ? 16u : 0u);
    }
  };
  for (int s = 0; s < G_AHEAD; s++) {
    if (s < nk) load(s, s);
    cp_async_commit();
  }
  constexpr uint32_t idesc = make_idesc(GM_T, GM_T);
  constexpr uint32_t sbo = (GK_T >> 3) * 128;
  bool ok = true;
  for (int kc = 0; kc < nk; kc++) {
    const int kb = kc + G_AHEAD;
    if (kb < nk) {
      const int s = kb % G_STAGES;
      if (kb >= G_STAGES) {
        // the MMAs of block kb - G_STAGES (issued at kc - 2) used this stage
        const bool got = mbar_wait(&mbar[s], (uint32_t)((kb / G_STAGES) - 1) & 1u, wait_limit);
        if (__syncthreads_or(!got)) {
          ok = false;
          break;
        }
      }
      load(kb, s);
    }
    cp_async_commit();
    cp_async_wait<G_AHEAD>();
    fence_async_smem();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t st = sbase + (uint32_t)(kc % G_STAGES) * G_STAGE;
#pragma unroll
      for (int kk = 0; kk < GK_T / 16; kk++) {
        const uint32_t ko = (uint32_t)kk * 256u;
        const uint64_t ah = make_desc(st + ko, 128, sbo), al = make_desc(st + G_OPB + ko, 128, sbo);
        const uint64_t bh = make_desc(st + 2 * G_OPB + ko, 128, sbo),
                       bl = make_desc(st + 3 * G_OPB + ko, 128, sbo);
        mma_bf16(tmem, ah, bh, idesc, (kc | kk) ? 1u : 0u);
        mma_bf16(tmem, al, bh, idesc, 1u);
        mma_bf16(tmem, ah, bl, idesc, 1u);
      }
      mma_commit(&mbar[kc % G_STAGES]);
    }
  }
  cp_async_wait<0>();
  if (tid == 0) mma_commit(&mdone);
  bool done = ok && mbar_wait(&mdone, 0, wait_limit);
  if (__syncthreads_or(!done)) {
    if (tid == 0) atomicExch(err, MBE_ETIMEOUT);
    done = false;
    // the MMAs issued so far must end before the accumulator is released
    if (tid == 0) mbar_wait(&mdone, 0, SPIN_LIMIT);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done) {
    const int row = m0 + 32 * warp + lane;
    float* wr = W + (int64_t)b * w_stride + (int64_t)row * nstr;
    const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
    for (int cc = 0; cc < GM_T; cc += 16) {
      float v[16];
      tmem_ld8x2(ta + (uint32_t)cc, ta + (uint32_t)(cc + 8), v);
      if (row < nstr) {
#pragma unroll
        for (int j = 0; j < 16; j++)
          if (n0 + cc + j < nstr) wr[n0 + cc + j] = v[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// ------------------------------------------------------------ W += Z/2
// Persistent, warp-specialised.  Work item = (tuple b, string a); a step =
// (row a, tile t of 128 column strings b''):
//   warp 0 (one thread)  waits for the A stage, row a's B operand and a free
//                        TMEM accumulator, issues kl/16 x 3 MMAs (M = 128
//                        column strings, N = kp pairs Q, K = kl compacted
//                        links of a) and commits to the barriers that free
//                        the operands and fill the accumulator;
//   warps 1 - 4          A: rows J_a(P_i) of c (hi and lo), the columns of
//                        tile t, cp.async into an MN-major stage (core
//                        matrix = 8 links x 8 column strings); one warp per
//                        stage (2 to 4 stages), each taking the steps of its
//                        stage, so that every stage has its copies in flight
//                        at once; rows i >= n_link stay zero;
//   warp 5               B, once per row a: rows P_i of g'/2 (from global
//                        memory), sign s_a(P_i) applied by an XOR of the bf16
//                        sign bits, MN-major, double-buffered across rows;
//   warps 6 - 21         copy the accumulator F^T (TMEM lanes = column
//                        strings b'', columns = pairs Q; four warps per lane
//                        quadrant, a quarter of the columns each) to shared
//                        memory and release it; then every thread adds, for
//                        each string J it owns (J = thread + 512 k), the
//                        entries that reach J:  W(a, J) += sum s F(b'', Q)
//                        over the links (Q, b'') of J with b'' in the tile
//                        (L_Q is symmetric: the column strings that feed J
//                        through Q are exactly J's own links; the lists, per
//                        string and tile, sit in shared memory when they fit).
//                        The sums of a row collect in shared memory (each
//                        thread owns its strings) and are added to W(a, :)
//                        (which holds H^a c) at the end of the row: no
//                        atomics, a fixed summation order.
// Every wait is bounded (wait_limit polls, each suspending the thread for at
// most AB_HINT_NS); a role that gives up sets the CTA's abort flag and the
// error word, the others leave their loops, the MMA thread waits for its own
// MMAs before the accumulators are freed.
constexpr int AB_M = 128;
constexpr int AB_MAX_STAGES = 4;                 // A stages = A copy warps 1..4
constexpr int AB_BWARP = 1 + AB_MAX_STAGES;      // warp 5 builds B
constexpr int AB_EPI0 = AB_BWARP + 1;            // first epilogue warp
constexpr int AB_EPI_WARPS = 16;
constexpr int AB_EPI_THREADS = AB_EPI_WARPS * 32;
constexpr int AB_THREADS = (AB_EPI0 + AB_EPI_WARPS) * 32;
constexpr int AB_NSTR_MAX = 8192;
constexpr uint32_t AB_HINT_NS = 1000;
// sleep caps of the waiting roles: the producers and the MMA thread wait for
// steps ahead (up to 256 ns between polls); the epilogue's poller is on the
// critical path (64 ns)
constexpr uint32_t AB_SLEEP_PROD = 256, AB_SLEEP_EPI = 64;

struct AbLayout {
  uint32_t a, b, f, acc, pl, po, total, a_bytes, b_bytes;
  int fs;                              // row stride of the staged F tile (floats)
  int pull_smem;                       // 1: the pull lists are staged in shared memory
  int ng;                              // epilogue groups (1 or 2)
};

__host__ __device__ inline AbLayout ab_layout(int kp, int kl, int nst, int nstr, int nlink,
                                              int pull_smem, int ng) {
  AbLayout L;
  uint32_t o = 0;
  auto take = [&](uint32_t bytes) {
    const uint32_t r = o;
    o += (bytes + 1023u) & ~1023u;
    return r;
  };
  const int ntiles = (nstr + AB_M - 1) / AB_M;
  L.a_bytes = (uint32_t)kl * AB_M * 2 * 2;
  L.b_bytes = (uint32_t)kl * kp * 2 * 2;
  L.fs = kp + 4;
  L.pull_smem = pull_smem;
  L.ng = ng;
  L.a = take(L.a_bytes * nst);
  L.b = take(L.b_bytes * 2);
  L.f = take((uint32_t)AB_M * L.fs * 4 * ng);   // one staged tile per epilogue group
  L.acc = take((uint32_t)nstr * 4 * 2);         // row sums of the even and odd tiles
  L.pl = pull_smem ? take((uint32_t)nstr * nlink * 2) : o;
  L.po = pull_smem ? take((uint32_t)nstr * (ntiles + 1) * 4) : o;
  L.total = o + 1024;   // alignment slack of the dynamic window
  return L;
}

// compacted links of every string: one warp per string, entries
// (J << 8) | (P << 1) | (sign < 0) for the pairs P with a link, ascending
__global__ void k_link_compact(const int32_t* __restrict__ link, int nstr, int npair, int nlink,
                               int32_t* __restrict__ lnk) {
  const int lane = threadIdx.x & 31;
  const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (a >= nstr) return;
  int n = 0;
  for (int p0 = 0; p0 < npair; p0 += 32) {
    const int P = p0 + lane;
    const int t = P < npair ? link[(int64_t)a * npair + P] : -1;
    const unsigned m = __ballot_sync(0xffffffffu, t >= 0);
    const int pos = n + __popc(m & ((1u << lane) - 1u));
    if (t >= 0 && pos < nlink) lnk[(int64_t)a * nlink + pos] = ((t >> 1) << 8) | (P << 1) | (t & 1);
    n += __popc(m);
  }
}

// the pull lists of the scatter: for string J, its links (Q, b'') ordered by
// the tile of b'' (stable in Q), each as the word offset of F(b'' mod 128, Q)
// in the staged tile (row stride fs) with the sign in bit 15; poff[J][t] is
// the first entry of tile t (poff[J][ntiles] = nlink).  One warp per string.
__global__ void k_pull_tables(const int32_t* __restrict__ lnk, int nstr, int nlink, int ntiles,
                              int fs, int16_t* __restrict__ plist, int32_t* __restrict__ poff) {
  const int lane = threadIdx.x & 31;
  const int J = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (J >= nstr) return;
  const int32_t* lr = lnk + (int64_t)J * nlink;
  const int e0 = lane < nlink ? lr[lane] : -1, e1 = lane + 32 < nlink ? lr[lane + 32] : -1;
  const int t0 = e0 >= 0 ? (e0 >> 8) >> 7 : -1, t1 = e1 >= 0 ? (e1 >> 8) >> 7 : -1;
  int n = 0;
  for (int t = 0; t < ntiles; t++) {
    if (lane == 0) poff[(int64_t)J * (ntiles + 1) + t] = n;
    const unsigned m0 = __ballot_sync(0xffffffffu, t0 == t), m1 = __ballot_sync(0xffffffffu, t1 == t);
    const unsigned below = (1u << lane) - 1u;
    if (t0 == t) {
      const int pos = n + __popc(m0 & below);
      const int bl = (e0 >> 8) & 127, Q = (e0 >> 1) & 127;
      plist[(int64_t)J * nlink + pos] = (int16_t)((bl * fs + Q) | ((e0 & 1) << 15));
    }
    if (t1 == t) {
      const int pos = n + __popc(m0) + __popc(m1 & below);
      const int bl = (e1 >> 8) & 127, Q = (e1 >> 1) & 127;
      plist[(int64_t)J * nlink + pos] = (int16_t)((bl * fs + Q) | ((e1 & 1) << 15));
    }
    n += __popc(m0) + __popc(m1);
  }
  if (lane == 0) poff[(int64_t)J * (ntiles + 1) + ntiles] = n;
}

// entry i (< nlink <= 64) of a string's compacted link list held as two
// registers per lane (e0: entries 0-31, e1: 32-63); all lanes take part
__device__ __forceinline__ int link_entry(int e0, int e1, int i) {
  const int s0 = __shfl_sync(0xffffffffu, e0, i & 31);
  const int s1 = __shfl_sync(0xffffffffu, e1, i & 31);
  return i < 32 ? s0 : s1;
}

template <int KP, bool PULL_SMEM, int NG>
__global__ void __launch_bounds__(AB_THREADS, 1)
k_sigma_ab(const int32_t* __restrict__ lnk, const int16_t* __restrict__ plist,
           const int32_t* __restrict__ poff, int nstr, int nlink, int kl,
           const bf16* __restrict__ gh, const bf16* __restrict__ cs, int64_t cs_stride, int ldc,
           const int32_t* __restrict__ active, int B, int nst, float* __restrict__ W,
           int64_t w_stride, long long wait_limit, int32_t* __restrict__ err) {
  constexpr int pull_smem = PULL_SMEM ? 1 : 0;
  extern __shared__ uint8_t dsm[];
  uint8_t* sm = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  __shared__ uint64_t full_a[AB_MAX_STAGES], empty_a[AB_MAX_STAGES], full_b[2], empty_b[2],
      acc_full[2], acc_empty[2], mdone;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  const AbLayout L = ab_layout(KP, kl, nst, nstr, nlink, pull_smem, NG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nitems = B * nstr, ntiles = (nstr + AB_M - 1) / AB_M;
  volatile int* abort_v = &abort_sh;

  // zero the operand stages (rows i >= nlink are never written); stage the
  // pull lists
  for (uint32_t i = tid; i < L.f / 16; i += AB_THREADS)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (pull_smem) {
    int16_t* spl = reinterpret_cast<int16_t*>(sm + L.pl);
    int32_t* spo = reinterpret_cast<int32_t*>(sm + L.po);
    for (int i = tid; i < nstr * nlink; i += AB_THREADS) spl[i] = plist[i];
    for (int i = tid; i < nstr * (ntiles + 1); i += AB_THREADS) spo[i] = poff[i];
  }
  if (warp == 0) tmem_alloc(&tmem_sh, 256);
  if (tid == 0) {
    for (int s = 0; s < AB_MAX_STAGES; s++) {
      mbar_init(&full_a[s], 1);
      mbar_init(&empty_a[s], 1);
    }
    for (int s = 0; s < 2; s++) {
      mbar_init(&full_b[s], 1);
      mbar_init(&empty_b[s], 1);
      mbar_init(&acc_full[s], 1);
      mbar_init(&acc_empty[s], AB_EPI_WARPS / NG);
    }
    mbar_init(&mdone, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;

  if (warp == 0) {
    // ------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = make_idesc_mn(AB_M, KP);
      const uint32_t a_lbo = (AB_M / 8) * 128, b_lbo = (uint32_t)(KP / 8) * 128;
      const uint32_t a_lo = (uint32_t)kl * AB_M * 2, b_lo = (uint32_t)kl * KP * 2;
      uint32_t j = 0, ir = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int b = item / nstr;
        if (active && !active[b]) continue;
        const int sbb = (int)(ir & 1u);
        const uint32_t pbb = (ir >> 1) & 1u;
        ok = mbar_wait_or_abort(&full_b[sbb], pbb, wait_limit, abort_v, AB_HINT_NS, AB_SLEEP_PROD);
        if (!ok) break;
        const uint32_t bb = smem_u32(sm + L.b + (uint32_t)sbb * L.b_bytes);
        for (int t = 0; t < ntiles; t++, j++) {
          const int sa = (int)(j % (uint32_t)nst), sb = (int)(j & 1u);
          const uint32_t pa = (j / (uint32_t)nst) & 1u, pb = (j >> 1) & 1u;
          ok = mbar_wait_or_abort(&full_a[sa], pa, wait_limit, abort_v, AB_HINT_NS, AB_SLEEP_EPI) &&
               mbar_wait_or_abort(&acc_empty[sb], pb ^ 1u, wait_limit, abort_v, AB_HINT_NS,
                                  AB_SLEEP_EPI);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ab = smem_u32(sm + L.a + (uint32_t)sa * L.a_bytes);
          const uint32_t d = tmem + (uint32_t)sb * 128u;
          for (int kk = 0; kk < kl / 16; kk++) {
            const uint32_t ao = (uint32_t)kk * 2u * a_lbo, bo = (uint32_t)kk * 2u * b_lbo;
            const uint64_t ah = make_desc(ab + ao, a_lbo, 128), al = make_desc(ab + a_lo + ao, a_lbo, 128);
            const uint64_t bh = make_desc(bb + bo, b_lbo, 128), bl = make_desc(bb + b_lo + bo, b_lbo, 128);
            mma_bf16(d, ah, bh, idesc, kk > 0 ? 1u : 0u);
            mma_bf16(d, al, bh, idesc, 1u);
            mma_bf16(d, ah, bl, idesc, 1u);
          }
          mma_commit(&empty_a[sa]);
          mma_commit(&acc_full[sb]);
          if (t == ntiles - 1) mma_commit(&empty_b[sbb]);
        }
        ir++;
      }
      if (!ok) {
        *abort_v = 1;
        atomicExch(err, MBE_ETIMEOUT);
      }
      // every MMA issued here ends before the accumulators are freed
      mma_commit(&mdone);
      mbar_wait(&mdone, 0, SPIN_LIMIT);
    }
  } else if (warp <= AB_MAX_STAGES) {
    // ------------------------------------------------ A: rows of c
    // warp 1 + s owns stage s: the steps j = s, s + nst, ... (one warp per
    // stage keeps the uses of a stage in order)
    const int sa = warp - 1;
    uint32_t j = 0, u = 0;
    bool ok = sa < nst;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int b = item / nstr, a = item - b * nstr;
      if (active && !active[b]) continue;
      const bf16* csb = cs + (int64_t)b * cs_stride;
      const int32_t* lr = lnk + (int64_t)a * nlink;
      const int e0 = lane < nlink ? lr[lane] : 0, e1 = lane + 32 < nlink ? lr[lane + 32] : 0;
      for (int t = 0; t < ntiles; t++, j++) {
        if ((int)(j % (uint32_t)nst) != sa) continue;
        bool got = lane == 0 ? mbar_wait_or_abort(&empty_a[sa], (u & 1u) ^ 1u, wait_limit, abort_v,
                                                  AB_HINT_NS, AB_SLEEP_PROD)
                             : true;
        ok = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
        if (!ok) break;
        const uint32_t base = smem_u32(sm + L.a + (uint32_t)sa * L.a_bytes);
        const int b0 = t * AB_M;
        for (int g = 0; g * 8 < nlink; g++) {
          const int i = g * 8 + (lane & 7);
          const int ent = link_entry(e0, e1, i);
          if (i < nlink) {
            const int64_t rowoff = (int64_t)(ent >> 8) * ldc;
#pragma unroll
            for (int jq = 0; jq < 4; jq++) {
              const int jj = jq * 4 + (lane >> 3);
              const int col = b0 + jj * 8;
              const bool in = col < nstr;
              const uint32_t dst = base + (uint32_t)g * 2048u + (uint32_t)jj * 128u + (uint32_t)(i & 7) * 16u;
#pragma unroll
              for (int hl = 0; hl < 2; hl++)
                cp_async16(dst + (uint32_t)hl * (uint32_t)kl * 256u,
                           csb + (int64_t)hl * nstr * ldc + rowoff + (in ? col : 0), in ? 16u : 0u);
            }
          }
        }
        cp_async_commit();
        cp_async_wait<0>();
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_a[sa]);
        u++;
      }
    }
    cp_async_wait<0>();
    if (!ok && sa < nst && lane == 0) {
      *abort_v = 1;
      atomicExch(err, MBE_ETIMEOUT);
    }
  } else if (warp == AB_BWARP) {
    // ------------------------------------------------ B: signed rows of g'/2
    uint32_t ir = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int b = item / nstr, a = item - b * nstr;
      if (active && !active[b]) continue;
      const int32_t* lr = lnk + (int64_t)a * nlink;
      const int e0 = lane < nlink ? lr[lane] : 0, e1 = lane + 32 < nlink ? lr[lane + 32] : 0;
      const int sbb = (int)(ir & 1u);
      const uint32_t pbb = (ir >> 1) & 1u;
      bool got = lane == 0 ? mbar_wait_or_abort(&empty_b[sbb], pbb ^ 1u, wait_limit, abort_v,
                                                AB_HINT_NS, AB_SLEEP_PROD)
                           : true;
      ok = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
      if (!ok) break;
      for (int g = 0; g * 8 < nlink; g++) {
        const int i = g * 8 + (lane & 7);
        const int ent = link_entry(e0, e1, i);
        if (i < nlink) {
          const uint32_t sgn = (ent & 1) ? 0x80008000u : 0u;
#pragma unroll
          for (int hl = 0; hl < 2; hl++) {
            const bf16* srow = gh + (((int64_t)b * 2 + hl) * KP + ((ent >> 1) & 127)) * KP;
            uint8_t* drow = sm + L.b + (uint32_t)sbb * L.b_bytes +
                            (uint32_t)hl * (uint32_t)kl * KP * 2u + (uint32_t)g * (KP * 16) +
                            (uint32_t)(i & 7) * 16u;
#pragma unroll
            for (int qq = 0; qq < (KP / 8 + 3) / 4; qq++) {
              const int qb = qq * 4 + (lane >> 3);
              if (qb < KP / 8) {
                uint4 v = *reinterpret_cast<const uint4*>(srow + qb * 8);
                v.x ^= sgn;
                v.y ^= sgn;
                v.z ^= sgn;
                v.w ^= sgn;
                *reinterpret_cast<uint4*>(drow + qb * 128) = v;
              }
            }
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_b[sbb]);
      ir++;
    }
    if (!ok && lane == 0) {
      *abort_v = 1;
      atomicExch(err, MBE_ETIMEOUT);
    }
  } else {
    // ------------------------------------------------ stage F, pull into W
    // NG groups of the epilogue warps take the steps in turn (with two, group
    // g the steps j with j % 2 == g, i.e. accumulator g), each with its own
    // staged tile and row sums, so that one group's staging and pull overlap
    // the other's
    constexpr int GW = AB_EPI_WARPS / NG, GT = GW * 32;
    constexpr int NC = KP * NG / 4;            // pair columns staged per thread
    const int e = warp - AB_EPI0, g = e / GW, eg = e % GW;
    const int q = warp & 3, h = eg >> 2;
    const int col0 = h * NC;
    const int et = tid - (AB_EPI0 + g * GW) * 32;   // thread within the group
    float* sF = reinterpret_cast<float*>(sm + L.f) + g * AB_M * L.fs;
    // the row's sums over its even and its odd tiles are kept apart and added
    // at the end of the row (the same order whatever the group count)
    float* sAccB = reinterpret_cast<float*>(sm + L.acc);
    const int16_t* PL = PULL_SMEM ? reinterpret_cast<const int16_t*>(sm + L.pl) : plist;
    const int32_t* PO = PULL_SMEM ? reinterpret_cast<const int32_t*>(sm + L.po) : poff;
    float* frow = sF + (32 * q + lane) * L.fs + col0;
    uint32_t j = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
      const int b = item / nstr, a = item - b * nstr;
      if (active && !active[b]) continue;
      // this group's first step in the row (steps alternate between groups)
      const int t0 = NG == 1 ? 0 : (int)(((uint32_t)g - j) & 1u);
      for (int t = t0; t < ntiles && ok; t += NG) {
        const uint32_t jj = j + (uint32_t)t;
        const int sb = (int)(jj & 1u);
        const uint32_t pb = (jj >> 1) & 1u;
        // one thread waits for the accumulator; the group's others block in
        // the group barrier, which also tells that every thread of the group
        // has finished its previous pull (the staged tile may be overwritten)
        const bool got = et == 0 ? mbar_wait_or_abort(&acc_full[sb], pb, wait_limit, abort_v,
                                                      AB_HINT_NS, AB_SLEEP_EPI)
                                 : true;
        if (bar_red_or(1 + g, GT, !got)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)sb * 128u + (uint32_t)col0;
#pragma unroll
        for (int c = 0; c < NC; c += 8) {
          uint32_t v[8];
          if (c + 8 <= NC) {
            tmem_ld8_nowait(ta + (uint32_t)c, v);
          } else {
            tmem_ld4_nowait(ta + (uint32_t)c, v);
            v[4] = v[5] = v[6] = v[7] = 0u;
          }
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 8; k++) asm volatile("" : "+r"(v[k]));
          *reinterpret_cast<uint4*>(frow + c) = make_uint4(v[0], v[1], v[2], v[3]);
          if (c + 8 <= NC)
            *reinterpret_cast<uint4*>(frow + c + 4) = make_uint4(v[4], v[5], v[6], v[7]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[sb]);
        bar_sync_n(1 + g, GT);
        // pull: W(a, J) += sum over the links of J into this tile, for J >= a
        // only (Z is symmetric: the lower triangle comes from the transpose)
        float* sAcc = sAccB + (NG == 1 ? (t & 1) : g) * nstr;
        const bool first = NG == 1 ? t < 2 : t == t0;
        for (int J = a + et; J < nstr; J += GT) {
          const int32_t* po = PO + J * (ntiles + 1) + t;
          const int lo = po[0], hi = po[1];
          const int16_t* pl = PL + J * nlink;
          float s0 = 0.f, s1 = 0.f;
          int x = lo;
          if ((x & 1) && x < hi) {
            const int en = pl[x++];
            s1 += __int_as_float(__float_as_int(sF[en & 0x7FFF]) ^ ((en & 0x8000) << 16));
          }
          // two entries per 32-bit load where the pair is 4-byte aligned
          // (an even nlink and an even x); otherwise one at a time
          if (!(nlink & 1)) {
            for (; x + 2 <= hi; x += 2) {
              const uint32_t pr = *reinterpret_cast<const uint32_t*>(pl + x);
              const float f0 = sF[pr & 0x7FFFu], f1 = sF[(pr >> 16) & 0x7FFFu];
              s0 += __int_as_float(__float_as_int(f0) ^ ((pr & 0x8000u) << 16));
              s1 += __int_as_float(__float_as_int(f1) ^ (pr & 0x80000000u));
            }
          }
          for (; x < hi; x++) {
            const int en = pl[x];
            s0 += __int_as_float(__float_as_int(sF[en & 0x7FFF]) ^ ((en & 0x8000) << 16));
          }
          const float s = s0 + s1;
          sAcc[J] = first ? s : sAcc[J] + s;
        }
      }
      j += (uint32_t)ntiles;
      // two groups meet at the end of the row (also after a failed wait, so
      // that neither is left waiting for the other); one group's threads
      // already agree (its barrier), and each reads only the sums it wrote
      if (NG == 2) {
        if (bar_red_or(3, AB_EPI_THREADS, !ok)) {
          ok = false;
          break;
        }
      } else if (!ok) {
        break;
      }
      // F carries g'/2: the upper triangle takes Z(a, J) = 2 (F pulled), the
      // diagonal Z(a, a) / 2, so that sigma = W + W^T holds Z once; the two
      // groups' sums of each J are added by one thread of either group
      const bool two = ntiles > 1;                      // odd tiles summed too
      // the array of the even tiles: 0, or the group that had step t = 0
      const int ev = NG == 1 ? 0 : (int)((j - (uint32_t)ntiles) & 1u);
      float* wr = W + (int64_t)b * w_stride + (int64_t)a * nstr;
      for (int J = a + e * 32 + lane; J < nstr; J += AB_EPI_THREADS) {
        float v = sAccB[ev * nstr + J];
        if (two) v += sAccB[(ev ^ 1) * nstr + J];
        wr[J] += J > a ? 2.f * v : v;
      }
      // the sums are read before either group overwrites them in the next row
      if (NG == 2) bar_sync_n(3, AB_EPI_THREADS);
    }
    if (!ok && et == 0) {
      *abort_v = 1;
      atomicExch(err, MBE_ETIMEOUT);
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// sigma(a,b) = W(a,b) + W(b,a) + shift (S^2 c)(a,b), FP32 output.  For
// Ms = 0, S^2 = S- S+ gives (S^2 c)(a, b) = (n_sigma - |a & b|) c(a, b) -
// sum over q in a\b, p in b\a of the signed c(a - q + p, b - p + q).
// sigma is symmetric: one CTA per 32 x 32 tile pair (I, J), I <= J, forms
// the values of tile (I, J) once (the spin term's gathers of c are the cost
// of this kernel) and writes them to both tiles, the transpose through
// shared memory so that every store is coalesced.  packed: c and sigma in
// the packed symmetric layout (sym_index), only tile (I, J) is written.
__global__ void k_sigma_tc_finish(const float* __restrict__ X, int64_t x_stride,
                                  const int32_t* __restrict__ link, const uint32_t* __restrict__ masks,
                                  int nstr, int n, int nsig, const float* __restrict__ c,
                                  int64_t c_stride, float shift, const int32_t* __restrict__ active,
                                  float* __restrict__ out, int64_t out_stride, int packed) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nt = (nstr + 31) / 32;
  int t = blockIdx.x, I = 0;
  while (t >= nt - I) {
    t -= nt - I;
    I++;
  }
  const int J = I + t;
  __shared__ float sX[2][32][33];
  const float* Xb = X + (int64_t)b * x_stride;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  // sX[0] = tile (I, J) of W, sX[1] = tile (J, I)
  for (int h = 0; h < 2; h++) {
    const int r0 = (h ? J : I) * 32, c0 = (h ? I : J) * 32;
    for (int i = ty; i < 32; i += ny) {
      const int row = r0 + i, col = c0 + tx;
      sX[h][i][tx] = (row < nstr && col < nstr) ? Xb[(int64_t)row * nstr + col] : 0.f;
    }
  }
  __syncthreads();
  const int npair = n * (n + 1) / 2;
  const float* cb = c + (int64_t)b * c_stride;
  float* ob = out + (int64_t)b * out_stride;
  float v[4];
  for (int k = 0, i = ty; i < 32; i += ny, k++) {
    const int ia = I * 32 + i, ib = J * 32 + tx;    // element (ia, ib) and its transpose
    float s = sX[0][i][tx] + sX[1][tx][i];
    if (shift != 0.f && ia < nstr && ib < nstr) {
      // evaluated for (min, max): on the diagonal tile both elements of a
      // pair get bitwise the same value
      const int lo = min(ia, ib), hi = max(ia, ib);
      const int32_t* la = link + (int64_t)lo * npair;
      const int32_t* lb = link + (int64_t)hi * npair;
      const uint32_t ma = masks[lo], mb = masks[hi];
      float s2 = (float)(nsig - __popc(ma & mb)) *
                 cb[packed ? sym_index(lo, hi, nstr) : (int64_t)lo * nstr + hi];
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
          const float x = cb[packed ? sym_index(ta >> 1, tb >> 1, nstr)
                                    : (int64_t)(ta >> 1) * nstr + (tb >> 1)];
          s2 -= ((ta ^ tb) & 1) ? -x : x;
        }
      }
      s += shift * s2;
    }
    v[k] = s;
    if (ia < nstr && ib < nstr) {
      if (!packed)
        ob[(int64_t)ia * nstr + ib] = s;
      else if (ia <= ib)
        ob[sym_index(ia, ib, nstr)] = s;
    }
  }
  if (I == J || packed) return;                      // the tile was its own transpose
  __syncthreads();
  for (int k = 0, i = ty; i < 32; i += ny, k++) sX[0][i][tx] = v[k];
  __syncthreads();
  for (int i = ty; i < 32; i += ny) {
    const int ia = J * 32 + i, ib = I * 32 + tx;
    if (ia < nstr && ib < nstr) ob[(int64_t)ia * nstr + ib] = sX[0][tx][i];
  }
}

struct AbPlan {
  int kp, nlink, kl, ldc, nst;
  AbLayout L;
};

// dynamic shared memory of k_sigma_ab: 227 KB per CTA less its static
// barriers
constexpr uint32_t AB_SMEM_MAX = 224 * 1024;

// operand plan of k_sigma_ab, the first that fits of: the pull lists in
// shared memory with 4, then 3 A stages (two epilogue groups before one),
// the lists in global memory likewise, then 2 stages.  Measured on the
// order-6 bins of the 8e/23o workload (autotuner, 64 tuples): for 8e/12o the
// lists in shared memory matter most (one group, 4 stages, lists in shared
// memory 1.24 ms; two groups only fit with the lists in global memory,
// 1.28 ms at best); for 6e/12o, where both fit, two groups win (0.25 against
// 0.32 ms)
inline bool ab_plan(int n, int nsig, int nstr, AbPlan& p) {
  const int npair = n * (n + 1) / 2;
  p.kp = round_up(npair, 16);
  p.nlink = nsig * (n - nsig + 1);
  p.kl = round_up(std::max(p.nlink, 1), 16);
  p.ldc = round_up(nstr, 8);
  if (p.kp > 128 || p.kl > 64 || nstr > AB_NSTR_MAX) return false;
  static const int order[][3] = {  // {pull lists in shared memory, stages, groups}
      {1, 4, 2}, {1, 4, 1}, {1, 3, 2}, {1, 3, 1}, {0, 4, 2}, {0, 3, 2}, {0, 4, 1},
      {0, 3, 1}, {1, 2, 2}, {1, 2, 1}, {0, 2, 2}, {0, 2, 1}};
  for (const auto& o : order) {
    p.nst = o[1];
    p.L = ab_layout(p.kp, p.kl, p.nst, nstr, p.nlink, o[0], o[2]);
    if (p.L.total <= AB_SMEM_MAX) return true;
  }
  return false;
}

// a given operand plan (nst A stages, pull lists in shared memory or not, ng
// epilogue groups), if its layout fits
inline bool ab_plan_with(int n, int nsig, int nstr, int nst, int ps, int ng, AbPlan& p) {
  if (!ab_plan(n, nsig, nstr, p)) return false;
  if (nst < 2 || nst > AB_MAX_STAGES || ng < 1 || ng > 2) return false;
  p.nst = nst;
  p.L = ab_layout(p.kp, p.kl, p.nst, nstr, p.nlink, ps, ng);
  return p.L.total <= AB_SMEM_MAX && p.L.pull_smem == (ps != 0);
}

template <int KP, bool PS, int NG>
void launch_ab_kps(int device, int grid, const AbPlan& p, cudaStream_t st, const int32_t* lnk,
                   const int16_t* plist, const int32_t* poff, int nstr, const bf16* gh,
                   const bf16* cs, int64_t cs_stride, const int32_t* active, int B, float* W,
                   int64_t w_stride, long long wait_limit, int32_t* err) {
  static bool attr_done[MBE_MAX_DEVICES] = {false};
  once_per_device(attr_done, device, [] {
    CU_CHECK(cudaFuncSetAttribute(k_sigma_ab<KP, PS, NG>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AB_SMEM_MAX));
  });
  k_sigma_ab<KP, PS, NG><<<grid, AB_THREADS, p.L.total, st>>>(
      lnk, plist, poff, nstr, p.nlink, p.kl, gh, cs, cs_stride, p.ldc, active, B, p.nst, W,
      w_stride, wait_limit, err);
}

template <int KP>
void launch_ab_kp(int device, int grid, const AbPlan& p, cudaStream_t st, const int32_t* lnk,
                  const int16_t* plist, const int32_t* poff, int nstr, const bf16* gh,
                  const bf16* cs, int64_t cs_stride, const int32_t* active, int B, float* W,
                  int64_t w_stride, long long wait_limit, int32_t* err) {
#define MBE_AB_KPS(PS, NG)                                                                \
  launch_ab_kps<KP, PS, NG>(device, grid, p, st, lnk, plist, poff, nstr, gh, cs, cs_stride, \
                            active, B, W, w_stride, wait_limit, err)
  if (p.L.ng == 2) {
    if (p.L.pull_smem) MBE_AB_KPS(true, 2);
    else MBE_AB_KPS(false, 2);
  } else {
    if (p.L.pull_smem) MBE_AB_KPS(true, 1);
    else MBE_AB_KPS(false, 1);
  }
#undef MBE_AB_KPS
}

void launch_ab(int device, int grid, const AbPlan& p, cudaStream_t st, const int32_t* lnk,
               const int16_t* plist, const int32_t* poff, int nstr, const bf16* gh, const bf16* cs,
               int64_t cs_stride, const int32_t* active, int B, float* W, int64_t w_stride,
               long long wait_limit, int32_t* err) {
  switch (p.kp) {
#define MBE_AB_CASE(KP)                                                                     \
  case KP:                                                                                  \
    launch_ab_kp<KP>(device, grid, p, st, lnk, plist, poff, nstr, gh, cs, cs_stride, active, \
                     B, W, w_stride, wait_limit, err);                                      \
    break;
    MBE_AB_CASE(16)
    MBE_AB_CASE(32)
    MBE_AB_CASE(48)
    MBE_AB_CASE(64)
    MBE_AB_CASE(80)
    MBE_AB_CASE(96)
    MBE_AB_CASE(112)
    MBE_AB_CASE(128)
#undef MBE_AB_CASE
    default:
      throw MbeError{MBE_EINVAL, "unsupported pair padding for the tensor-core sigma"};
  }
}

int sm_count(int device) {
  static int cnt[MBE_MAX_DEVICES] = {0};
  static bool done[MBE_MAX_DEVICES] = {false};
  once_per_device(done, device, [&] {
    CU_CHECK(cudaDeviceGetAttribute(&cnt[device], cudaDevAttrMultiProcessorCount, device));
  });
  return cnt[device];
}

}  // namespace

bool sigma_tc_supported(int n, int nstr) {
  if (n < 1 || n > 15) return false;
  AbPlan p;
  // the operand sizes grow with the link count: any electron count fits iff
  // the one with the most links does
  for (int nsig = 0; nsig <= n; nsig++)
    if (!ab_plan(n, nsig, nstr, p)) return false;
  return true;
}

void sigma_tc(mbe_ctx* ctx, BinProblem& bp, SigmaWork& w, const float* c, int64_t c_stride,
              float* out, int64_t out_stride, const int32_t* active, double spin_shift,
              bool packed) {
  const int npair = bp.npair, nstr = bp.nstr, B = bp.B;
  const int nsm = sm_count(ctx->device);
  AbPlan p;
  if (!ab_plan(bp.n, bp.nsig, nstr, p))
    throw MbeError{MBE_EINVAL, "active space too large for the tensor-core sigma"};
  // autotuned plan of this shape, if one is known
  bool tune_now = false;
  if (ctx->opt.autotune && p.nlink > 0) {
    auto it = ctx->tune_ab.find({bp.n, bp.nsig});
    AbPlan q;
    if (it == ctx->tune_ab.end())
      tune_now = true;
    else if (ab_plan_with(bp.n, bp.nsig, nstr, it->second[0], it->second[1], it->second[2], q))
      p = q;
  }
  const int64_t N = bp.ndet;
  const int64_t hs = 2 * (int64_t)nstr * p.ldc;      // bf16 elements per tuple (hi + lo)
  const int ntiles = (nstr + AB_M - 1) / AB_M;
  cudaStream_t st = ctx->stream;
  // per bin shape: compacted links and the pull lists of the scatter
  StringTables* tab = get_tables(ctx, bp.n, bp.nsig);
  if (tab->nlink != p.nlink) {
    tab->lnk.reset(&ctx->pool, (size_t)nstr * std::max(p.nlink, 1));
    tab->plist.reset(&ctx->pool, (size_t)nstr * std::max(p.nlink, 1));
    tab->poff.reset(&ctx->pool, (size_t)nstr * (ntiles + 1));
    tab->nlink = p.nlink;
    if (p.nlink > 0) {
      k_link_compact<<<(nstr + 7) / 8, 256, 0, st>>>(tab->link.ptr, nstr, npair, p.nlink,
                                                      tab->lnk.ptr);
      CU_LAUNCH_CHECK();
      k_pull_tables<<<(nstr + 7) / 8, 256, 0, st>>>(tab->lnk.ptr, nstr, p.nlink, ntiles, p.L.fs,
                                                     tab->plist.ptr, tab->poff.ptr);
      CU_LAUNCH_CHECK();
    }
  }
  if (w.Xf.n < (size_t)B * N) w.Xf.reset(&ctx->pool, (size_t)B * N);
  // the timeout word is cleared once, when it is allocated: a timeout of
  // any call of the batch stays visible to sigma_tc_error
  if (!w.err.ptr) {
    w.err.reset(&ctx->pool, 1);
    CU_CHECK(cudaMemsetAsync(w.err.ptr, 0, sizeof(int32_t), st));
  }
  if (w.csplit.n < (size_t)B * hs * 2) w.csplit.reset(&ctx->pool, (size_t)B * hs * 2);
  // per batch (constant over the Davidson iteration): g'/2 split and H^a
  const size_t gbytes = (size_t)B * 2 * p.kp * p.kp * 2;
  if (bp.gsplit.n != gbytes) {
    bp.gsplit.reset(&ctx->pool, gbytes);
    k_prep_gh<<<dim3(8, B), 256, 0, st>>>(bp.gp.ptr, npair, p.kp, (bf16*)bp.gsplit.ptr);
    CU_LAUNCH_CHECK();
  }
  if (bp.haa.n != (size_t)B * hs * 2) {
    bp.haa.reset(&ctx->pool, (size_t)B * hs * 2);
    const int smem = (int)(sizeof(double) * nstr);
    static bool attr_done[MBE_MAX_DEVICES] = {false};
    once_per_device(attr_done, ctx->device, [] {
      CU_CHECK(cudaFuncSetAttribute(k_build_haa, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    64 * 1024));
    });
    if (smem > 64 * 1024) throw MbeError{MBE_EINVAL, "too many strings for the H^a build"};
    k_build_haa<<<dim3(nstr, B), HAA_THREADS, smem, st>>>(bp.tab->link.ptr, nstr, npair,
                                                          bp.gp.ptr, p.ldc, (bf16*)bp.haa.ptr, hs);
    CU_LAUNCH_CHECK();
  }
  bf16* cs = (bf16*)w.csplit.ptr;
  if (packed) {
    const int ntp = (nstr + 31) / 32;
    k_split_c_sym<<<dim3((unsigned)(ntp * (ntp + 1) / 2), B), 256, 0, st>>>(c, c_stride, nstr,
                                                                           p.ldc, active, cs, hs);
    CU_LAUNCH_CHECK();
  } else {
    const int64_t work = (int64_t)nstr * (p.ldc / 8);
    const unsigned gx = (unsigned)std::min<int64_t>((work + 255) / 256, 1024);
    k_split_c<<<dim3(gx, B), 256, 0, st>>>(c, c_stride, nstr, p.ldc, active, cs, hs);
    CU_LAUNCH_CHECK();
  }
  const long long wl = ctx->opt.wait_limit;
  const int nt_g = (nstr + GM_T - 1) / GM_T;
  const int grid_ab = (int)std::min<int64_t>((int64_t)B * nstr, nsm);
  if (tune_now) {
    // every plan that fits, timed on this call's data (H^a c rewritten
    // before each, so W ends correct whichever runs last); the best of two
    // timed launches per plan counts
    static bool attr_done[MBE_MAX_DEVICES] = {false};
    once_per_device(attr_done, ctx->device, [] {
      CU_CHECK(cudaFuncSetAttribute(k_gemm_haa, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)G_SMEM));
    });
    cudaEvent_t e0, e1;
    CU_CHECK(cudaEventCreate(&e0));
    CU_CHECK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_nst = p.nst, best_ps = p.L.pull_smem ? 1 : 0, best_ng = p.L.ng;
    for (int ng = 1; ng <= 2; ng++)
    for (int nst = 2; nst <= AB_MAX_STAGES; nst++)
      for (int ps = 0; ps <= 1; ps++) {
        AbPlan q;
        if (!ab_plan_with(bp.n, bp.nsig, nstr, nst, ps, ng, q)) continue;
        float t = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
          k_gemm_haa<<<dim3(nt_g * nt_g, B), G_THREADS, G_SMEM, st>>>(
              (const bf16*)bp.haa.ptr, cs, hs, nstr, p.ldc, active, w.Xf.ptr, N, wl, w.err.ptr);
          CU_LAUNCH_CHECK();
          CU_CHECK(cudaEventRecord(e0, st));
          launch_ab(ctx->device, grid_ab, q, st, tab->lnk.ptr, tab->plist.ptr, tab->poff.ptr,
                    nstr, (const bf16*)bp.gsplit.ptr, cs, hs, active, B, w.Xf.ptr, N, wl,
                    w.err.ptr);
          CU_LAUNCH_CHECK();
          CU_CHECK(cudaEventRecord(e1, st));
          CU_CHECK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CU_CHECK(cudaEventElapsedTime(&ms, e0, e1));
          if (rep > 0) t = std::min(t, ms);
        }
        if (ctx->opt.verbose)
          fprintf(stderr, "[mbe autotune] n=%d nsig=%d stages=%d pull_smem=%d groups=%d %.4f ms\n",
                  bp.n, bp.nsig, nst, ps, ng, t);
        if (t < best) {
          best = t;
          best_nst = nst;
          best_ps = ps;
          best_ng = ng;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune_ab[{bp.n, bp.nsig}] = {best_nst, best_ps, best_ng};
    AbPlan q;
    if (ab_plan_with(bp.n, bp.nsig, nstr, best_nst, best_ps, best_ng, q)) p = q;
    if (!ctx->tune_file.empty()) {
      std::ofstream out(ctx->tune_file, std::ios::app);
      out << "sigma_ab " << bp.n << " " << bp.nsig << " " << best_nst << " " << best_ps << " "
          << best_ng << " " << best << "\n";
    }
  }
  cudaEvent_t ev;
  ctx->dom_timer.begin(st, ctx->opt.timing != 0, &ev);
  {
    static bool attr_done[MBE_MAX_DEVICES] = {false};
    once_per_device(attr_done, ctx->device, [] {
      CU_CHECK(cudaFuncSetAttribute(k_gemm_haa, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)G_SMEM));
    });
    k_gemm_haa<<<dim3(nt_g * nt_g, B), G_THREADS, G_SMEM, st>>>(
        (const bf16*)bp.haa.ptr, cs, hs, nstr, p.ldc, active, w.Xf.ptr, N, wl, w.err.ptr);
    CU_LAUNCH_CHECK();
  }
  if (p.nlink > 0) {
    launch_ab(ctx->device, grid_ab, p, st, tab->lnk.ptr, tab->plist.ptr, tab->poff.ptr, nstr,
              (const bf16*)bp.gsplit.ptr, cs, hs, active, B, w.Xf.ptr, N, wl, w.err.ptr);
    CU_LAUNCH_CHECK();
  }
  ctx->dom_timer.end(st, ev);
  ctx->stats.dom_launches += 1;
  const int ntl = (nstr + 31) / 32;
  k_sigma_tc_finish<<<dim3((unsigned)(ntl * (ntl + 1) / 2), B), 256, 0, st>>>(w.Xf.ptr, N, bp.tab->link.ptr, bp.tab->masks.ptr,
                                                nstr, bp.n, bp.nsig, c, c_stride,
                                                (float)spin_shift, active, out, out_stride,
                                                packed ? 1 : 0);
  CU_LAUNCH_CHECK();
}

int32_t sigma_tc_error(mbe_ctx* ctx, SigmaWork& w) {
  if (!w.err.ptr) return 0;
  int32_t e = 0;
  CU_CHECK(cudaMemcpyAsync(&e, w.err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CU_CHECK(cudaStreamSynchronize(ctx->stream));
  return e;
}
