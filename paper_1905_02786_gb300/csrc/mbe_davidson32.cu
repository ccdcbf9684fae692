// Davidson iteration of the mixed-precision mode, laid out for GB300.
//
// GB300 issues FP64 arithmetic at roughly 1/60 of its FP32 rate, so every
// per-determinant operation here is FP32: the subspace vectors V, their
// sigma vectors AV, residuals and preconditioned corrections are stored and
// combined in FP32, with per-thread FP32 partial sums reduced in FP64 across
// threads.  FP64-grade quantities are formed only where the energy depends
// on them, at "exact points":
//   x      the current Ritz vector (FP32 values, taken as exact),
//   A x    by the FP64-grade sliced tensor-core contraction,
//   x.x    by an error-free FP32 dot (two-product + compensated sum),
//   theta  = x.Ax / x.x, the Rayleigh quotient reported as the energy,
//   r_x    = A x - theta x, its norm in FP64.
// Iteration (Davidson, J. Comput. Phys. 17, 87 (1975)):
//   stage A: tensor-core (split-BF16x3) sigma vectors until the residual is
//            below mixed_stage_tol max(1, |theta|) (default 1e-5, above
//            their precision floor);
//   rounds:  exact point; tuples with |r_x| above the target continue from
//            {x, t_1, ...} where t_j get tensor-core sigma vectors and the
//            couplings x.A t_j = theta (x.t_j) + r_x.t_j use only exact data;
//            the stage stops at max(target, mixed_round_drop |r_x|)
//            (default |r_x| / 100).
// The energy error of the reported Rayleigh quotient is below |r_x|^2 / gap.
#include "mbe_internal.cuh"
#include "mbe_ritz.cuh"
#include <algorithm>
#include <cmath>
#include <cstdio>

namespace {

constexpr int RT = 256;      // threads of the reduction kernels

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
  return s;
}

// Every FP32 vector of the mixed Davidson iteration is alpha-beta symmetric
// and kept packed (sym_index): L = sym_len(nstr) elements, about half of
// N_det, the padding kept at zero, each vector on a 16-byte boundary, so the
// streaming kernels below move float4s.  Their dot products weigh the
// float4s from nd4 = sym_nd / 4 on (the upper triangle) by 2, which gives
// the dot products of the full vectors.  A reduction chunk is `ch` elements
// (a multiple of 1024, chosen per batch).

__device__ __forceinline__ float dot4(const float4 a, const float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}

// partial[b][i][chunk] = sum over the chunk of w_k X[b][i][k] Y[b][k], i < m
__global__ void __launch_bounds__(RT) k32_multidot(const float* __restrict__ X, int64_t xb,
                                                  int64_t xv, const float* __restrict__ Y,
                                                  int64_t yb, int m, int64_t L, int64_t nd4, int ch,
                                                  int nchunks, const int32_t* __restrict__ active,
                                                  double* __restrict__ partial) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int chunk = blockIdx.x;
  const int64_t q0 = (int64_t)chunk * (ch >> 2), q1 = min(L >> 2, q0 + (ch >> 2));
  __shared__ double red[32][33];
  const float4* y = reinterpret_cast<const float4*>(Y + (int64_t)b * yb);
  const float* x = X + (int64_t)b * xb;
  for (int i0 = 0; i0 < m; i0 += 16) {
    const int ni = min(16, m - i0);
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; i++) acc[i] = 0.f;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      const float4 y0 = y[q];
      const float w = q < nd4 ? 1.f : 2.f;        // exact scaling
      const float4 yv = make_float4(w * y0.x, w * y0.y, w * y0.z, w * y0.w);
#pragma unroll
      for (int i = 0; i < 16; i++)
        if (i < ni)
          acc[i] = dot4(reinterpret_cast<const float4*>(x + (int64_t)(i0 + i) * xv)[q], yv, acc[i]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 16; i++) {
      double v = (double)acc[i];
      for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < ni) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w][threadIdx.x];
      partial[((int64_t)b * m + i0 + threadIdx.x) * nchunks + chunk] = s;
    }
    __syncthreads();
  }
}

// error-free dot of two FP32 vectors: products split exactly (p + e = x y),
// the p terms summed with compensation, all per-thread sums combined in FP64
__global__ void k32_dot_comp(const float* __restrict__ X, int64_t xb, const float* __restrict__ Y,
                             int64_t yb, int64_t N, int64_t nd, int ch, int nchunks,
                             const int32_t* __restrict__ active, double* __restrict__ partial) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ double red[32];
  const int64_t k0 = (int64_t)blockIdx.x * ch, k1 = min(N, k0 + ch);
  const float* x = X + (int64_t)b * xb;
  const float* y = Y + (int64_t)b * yb;
  // (s, lo): s + lo carries the running sum to ~2^-48 relative; every
  // product is split exactly (p + e = a b, fma) and every addition of p to s
  // exactly (TwoSum: s + p = t + err)
  float s = 0.f, lo = 0.f;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const float a = x[k] * (k < nd ? 1.f : 2.f), bb = y[k];   // weight: exact
    const float p = a * bb;
    const float e = fmaf(a, bb, -p);
    const float t = s + p;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (p - bp);
    s = t;
    lo += err + e;
  }
  const double tot = block_sum((double)s + (double)lo, red);
  if (threadIdx.x == 0) partial[(int64_t)b * nchunks + blockIdx.x] = tot;
}

__global__ void k32_final(const double* __restrict__ partial, int m, int nchunks,
                          const int32_t* __restrict__ active, double* __restrict__ out, int64_t ob,
                          int64_t oi) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double* p = partial + ((int64_t)b * m + i) * nchunks;
    double s = 0.0;
    for (int c = 0; c < nchunks; c++) s += p[c];
    out[(int64_t)b * ob + (int64_t)i * oi] = s;
  }
}

// G row j = m-1 from dots[b][i] (i < m); with exact0, entry 0 is replaced by
// theta_x (x.t_j) + r_x.t_j  (cdot = x.t_j error-free, rdot = r_x.t_j)
__global__ void k32_store_row(const double* __restrict__ dots, const double* __restrict__ cdot,
                              const double* __restrict__ rdot, const double* __restrict__ thx,
                              int m, int M, int exact0, const int32_t* __restrict__ active,
                              double* __restrict__ G) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  const int j = m - 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double v = dots[(int64_t)b * M + i];
    if (exact0 && i == 0 && j > 0) v = thx[b] * cdot[b] + rdot[b];
    G[(int64_t)b * M * M + (int64_t)j * M + i] = v;
    G[(int64_t)b * M * M + (int64_t)i * M + j] = v;
  }
}

// lowest eigenpair of the m x m subspace matrix G[b] (one warp per tuple)
__global__ void k32_jacobi(const double* __restrict__ G, int m, int M,
                          const int32_t* __restrict__ active, double* __restrict__ theta,
                          double* __restrict__ y) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  __shared__ RitzShared S;
  ritz_lowest(G + (int64_t)b * M * M, m, M, S, theta + b, y + (int64_t)b * M);
}

__global__ void k32_converge(const double* __restrict__ partial, int nchunks, int B, int it,
                             const double* __restrict__ tol_r, int rel,
                             const double* __restrict__ theta, double* __restrict__ rnorm,
                             int32_t* __restrict__ active, int32_t* __restrict__ iters,
                             int32_t* __restrict__ nactive) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (!active[b]) continue;
    double s = 0.0;
    for (int c = 0; c < nchunks; c++) s += partial[(int64_t)b * nchunks + c];
    const double rn = sqrt(s);
    rnorm[b] = rn;
    iters[b] += 1;
    const double tr = rel ? tol_r[b] * fmax(1.0, fabs(theta[b])) : tol_r[b];
    if (it > 0 && rn < tr) active[b] = 0;
    else atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *nactive = cnt;
}

// t = r / (theta - H_II) on the packed vector (the full vector's
// symmetrised correction: r and H_II are symmetric)
__global__ void k32_precondition(float* __restrict__ T, const float* __restrict__ hd, int64_t L,
                                 const double* __restrict__ theta,
                                 const int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const float th = (float)theta[b];
  float* Tb = T + (int64_t)b * L;
  const float* hb = hd + (int64_t)b * L;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < L;
       k += (int64_t)gridDim.x * blockDim.x) {
    float d = th - hb[k];
    if (fabsf(d) < 1e-4f) d = d < 0.f ? -1e-4f : 1e-4f;
    Tb[k] = Tb[k] / d;
  }
}

__global__ void k32_append(const float* __restrict__ T, float* __restrict__ V, int m, int M,
                           int64_t L, const double* __restrict__ nrm2,
                           int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const double n2 = nrm2[(int64_t)b * M];
  if (!(n2 > 1e-24)) {
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) active[b] = 2;
    return;
  }
  __shared__ float s_inv;
  if (threadIdx.x == 0) s_inv = (float)(1.0 / sqrt(n2));   // one FP64 root per block
  __syncthreads();
  const float inv = s_inv;
  const float4* t4 = reinterpret_cast<const float4*>(T + (int64_t)b * L);
  float4* v4 = reinterpret_cast<float4*>(V + (int64_t)b * M * L + (int64_t)m * L);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (L >> 2);
       q += (int64_t)gridDim.x * blockDim.x) {
    const float4 t = t4[q];
    v4[q] = make_float4(t.x * inv, t.y * inv, t.z * inv, t.w * inv);
  }
}

// Per-thread FP32 dot accumulators of the fused kernels below live in shared
// memory, sD[i][thread] (registers stay few and occupancy high: these kernels
// are bound by HBM).  Block sums of sD[i][.] for i < m, in FP64, go to
// partial[(b m + i) nchunks + chunk] (the layout of k32_multidot).
__device__ __forceinline__ void sd_sums_to_partial(const float (*sD)[RT], int m,
                                                   double* __restrict__ partial, int b,
                                                   int chunk, int nchunks) {
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < m; i += RT / 32) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < RT / 32; j++) v += (double)sD[i][lane + 32 * j];
    for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) partial[((int64_t)b * m + i) * nchunks + chunk] = v;
  }
}

// the same for pairs of accumulators: .x to partial, .y to partial2
__device__ __forceinline__ void sde_sums_to_partial(const float2 (*sDE)[RT], int m,
                                                    double* __restrict__ partial,
                                                    double* __restrict__ partial2, int b,
                                                    int chunk, int nchunks) {
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < m; i += RT / 32) {
    double v = 0.0, w = 0.0;
#pragma unroll
    for (int j = 0; j < RT / 32; j++) {
      const float2 a = sDE[i][lane + 32 * j];
      v += (double)a.x;
      w += (double)a.y;
    }
    for (int off = 16; off; off >>= 1) {
      v += __shfl_down_sync(0xffffffffu, v, off);
      w += __shfl_down_sync(0xffffffffu, w, off);
    }
    if (lane == 0) {
      partial[((int64_t)b * m + i) * nchunks + chunk] = v;
      partial2[((int64_t)b * m + i) * nchunks + chunk] = w;
    }
  }
}

// The residual step with the preconditioner and the first orthogonalisation
// pass's dot products folded in:
//   x = V y,  r = AV y - theta x (stage A), or with exact0
//   r = y_0 (r_x + (theta_x - theta) V_0) + sum_{i>=1} y_i (AV_i - theta V_i),
//   |r|^2 partials,
//   t = r / (theta - H_II)  (as k32_precondition),
//   partials of V_i . t, i < m.
// The second read of V_i[k] follows the first within the same thread and is
// served by the caches, so V streams from HBM once instead of twice.
__global__ void __launch_bounds__(RT) k32_residual_pre(
    const float* __restrict__ V, const float* __restrict__ AV, const float* __restrict__ RX,
    int exact0, int m, int M, int64_t L, int64_t nd4, const double* __restrict__ y,
    const double* __restrict__ theta, const double* __restrict__ thx,
    const float* __restrict__ hd, const int32_t* __restrict__ active, float* __restrict__ X,
    float* __restrict__ T, int ch, int nchunks, double* __restrict__ rpart,
    double* __restrict__ dpart, int olsen, float* __restrict__ Uo,
    double* __restrict__ upart, double* __restrict__ xpart) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  // per-thread dot accumulators: sD[i] for V_i . t, or with olsen sDE[i] for
  // (V_i . t, V_i . u) (one 8-byte shared access per vector and element)
  extern __shared__ float sdyn[];
  float (*sD)[RT] = reinterpret_cast<float (*)[RT]>(sdyn);
  float2 (*sDE)[RT] = reinterpret_cast<float2 (*)[RT]>(sdyn);
  __shared__ float sy[32];
  __shared__ double red[32];
  if (threadIdx.x < m) sy[threadIdx.x] = (float)y[(int64_t)b * M + threadIdx.x];
  for (int i = 0; i < m; i++) {
    if (olsen) sDE[i][threadIdx.x] = make_float2(0.f, 0.f);
    else sD[i][threadIdx.x] = 0.f;
  }
  __syncthreads();
  const float th = (float)theta[b];
  const float dth = exact0 ? (float)(thx[b] - theta[b]) : 0.f;
  const int i0 = exact0 ? 1 : 0;
  const int64_t Lq = L >> 2;
  const int64_t q0 = (int64_t)blockIdx.x * (ch >> 2), q1 = min(Lq, q0 + (ch >> 2));
  const float4* Vb = reinterpret_cast<const float4*>(V + (int64_t)b * M * L);
  const float4* AVb = reinterpret_cast<const float4*>(AV + (int64_t)b * M * L);
  const float4* hb = reinterpret_cast<const float4*>(hd + (int64_t)b * L);
  const float4* RXb = reinterpret_cast<const float4*>(RX + (int64_t)b * L);
  float4* Xb = reinterpret_cast<float4*>(X + (int64_t)b * L);
  float4* Tb = reinterpret_cast<float4*>(T + (int64_t)b * L);
  float4* Ub = olsen ? reinterpret_cast<float4*>(Uo + (int64_t)b * L) : nullptr;
  float acc = 0.f, xt = 0.f, xu = 0.f;
  for (int64_t q = q0 + threadIdx.x; q < q1; q += RT) {
    float xs[4] = {0.f, 0.f, 0.f, 0.f}, rs[4] = {0.f, 0.f, 0.f, 0.f};
    if (exact0) {
      const float4 v0 = Vb[q], rx = RXb[q];
      const float v[4] = {v0.x, v0.y, v0.z, v0.w}, r0[4] = {rx.x, rx.y, rx.z, rx.w};
#pragma unroll
      for (int e = 0; e < 4; e++) {
        xs[e] = sy[0] * v[e];
        rs[e] = sy[0] * (r0[e] + dth * v[e]);
      }
    }
#pragma unroll 4
    for (int i = i0; i < m; i++) {
      const float4 v4 = Vb[(int64_t)i * Lq + q], a4 = AVb[(int64_t)i * Lq + q];
      const float v[4] = {v4.x, v4.y, v4.z, v4.w}, a[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int e = 0; e < 4; e++) {
        xs[e] = fmaf(sy[i], v[e], xs[e]);
        rs[e] = fmaf(sy[i], a[e] - th * v[e], rs[e]);
      }
    }
    Xb[q] = make_float4(xs[0], xs[1], xs[2], xs[3]);
    const float4 h4 = hb[q];
    const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
    const float w = q < nd4 ? 1.f : 2.f;          // weight of the packed elements
    float ts[4], us[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
      acc = fmaf(w * rs[e], rs[e], acc);
      float d = th - hv[e];
      if (fabsf(d) < 1e-4f) d = d < 0.f ? -1e-4f : 1e-4f;
      ts[e] = rs[e] / d;
      us[e] = xs[e] / d;
    }
    const float4 t = make_float4(ts[0], ts[1], ts[2], ts[3]);
    const float4 tw = make_float4(w * ts[0], w * ts[1], w * ts[2], w * ts[3]);
    Tb[q] = t;
    if (olsen) {
      const float4 u = make_float4(us[0], us[1], us[2], us[3]);
      const float4 uw = make_float4(w * us[0], w * us[1], w * us[2], w * us[3]);
      Ub[q] = u;
#pragma unroll
      for (int e = 0; e < 4; e++) {
        xt = fmaf(w * xs[e], ts[e], xt);
        xu = fmaf(w * xs[e], us[e], xu);
      }
#pragma unroll 4
      for (int i = 0; i < m; i++) {
        const float4 v = Vb[(int64_t)i * Lq + q];
        float2 a = sDE[i][threadIdx.x];
        a.x = dot4(v, tw, a.x);
        a.y = dot4(v, uw, a.y);
        sDE[i][threadIdx.x] = a;
      }
    } else {
#pragma unroll 4
      for (int i = 0; i < m; i++)
        sD[i][threadIdx.x] = dot4(Vb[(int64_t)i * Lq + q], tw, sD[i][threadIdx.x]);
    }
  }
  const double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) rpart[(int64_t)b * nchunks + blockIdx.x] = tot;
  if (olsen) {
    __syncthreads();
    const double s_xt = block_sum((double)xt, red);
    if (threadIdx.x == 0) xpart[((int64_t)b * 2) * nchunks + blockIdx.x] = s_xt;
    __syncthreads();
    const double s_xu = block_sum((double)xu, red);
    if (threadIdx.x == 0) xpart[((int64_t)b * 2 + 1) * nchunks + blockIdx.x] = s_xu;
    sde_sums_to_partial(sDE, m, dpart, upart, b, blockIdx.x, nchunks);
  } else {
    sd_sums_to_partial(sD, m, dpart, b, blockIdx.x, nchunks);
  }
}

// Olsen's correction with the P-space preconditioner M = theta - A_0:
// t = M^-1 r - eps M^-1 x, eps = x.M^-1 r / x.M^-1 x (so that the exact
// block does not return t = -x).  From the reduced sums xsum[b] = (x.t1,
// x.u): eps[b], and with dots the first pass's coefficients
// V.t = V.t1 - eps V.u (coef holds V.t1, c2 V.u)
__global__ void k32_olsen(const double* __restrict__ xsum, const double* __restrict__ c2, int m,
                          int M, int dots, const int32_t* __restrict__ active,
                          double* __restrict__ coef, float* __restrict__ eps) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  const double xu = xsum[(int64_t)b * 2 + 1];
  double e = xsum[(int64_t)b * 2] / xu;
  if (!(xu != 0.0) || !isfinite(e)) e = 0.0;
  if (threadIdx.x == 0) eps[b] = (float)e;
  if (dots)
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      coef[(int64_t)b * M + i] -= e * c2[(int64_t)b * M + i];
}

// T <- T - eps U (Olsen's combination where the dots are taken afterwards)
__global__ void k32_sub_eps(float* __restrict__ T, const float* __restrict__ U,
                            const float* __restrict__ eps, int64_t N,
                            const int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const float e = eps[b];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    T[(int64_t)b * N + k] = fmaf(-e, U[(int64_t)b * N + k], T[(int64_t)b * N + k]);
}

// One classical Gram-Schmidt update T <- T - sum_{i<m} c_i V_i, with the dot
// products the next step needs taken in the same pass (V_i[k] read twice by
// one thread, the second time from the caches):
//   norm == 0: partials of V_i . T (the second pass's coefficients),
//   norm == 1: partials of T . T (the normalisation).
__global__ void __launch_bounds__(RT) k32_orth_pass(float* __restrict__ T,
                                                   const float* __restrict__ V, int m, int M,
                                                   int64_t L, int64_t nd4,
                                                   const double* __restrict__ coef,
                                                   const int32_t* __restrict__ active, int norm,
                                                   int ch, int nchunks, double* __restrict__ partial,
                                                   const float* __restrict__ Uo,
                                                   const float* __restrict__ eps) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ float sc[32];
  __shared__ float sD[32][RT];
  __shared__ double red[32];
  if (threadIdx.x < m) sc[threadIdx.x] = (float)coef[(int64_t)b * M + threadIdx.x];
  if (!norm)
    for (int i = 0; i < m; i++) sD[i][threadIdx.x] = 0.f;
  __syncthreads();
  const int64_t Lq = L >> 2;
  const int64_t q0 = (int64_t)blockIdx.x * (ch >> 2), q1 = min(Lq, q0 + (ch >> 2));
  const float4* Vb = reinterpret_cast<const float4*>(V + (int64_t)b * M * L);
  float4* Tb = reinterpret_cast<float4*>(T + (int64_t)b * L);
  float nacc = 0.f;
  // with Uo (first pass under Olsen's correction): T holds M^-1 r and the
  // update starts from t = M^-1 r - eps M^-1 x
  const float e = Uo ? eps[b] : 0.f;
  const float4* Ub = Uo ? reinterpret_cast<const float4*>(Uo + (int64_t)b * L) : nullptr;
  for (int64_t q = q0 + threadIdx.x; q < q1; q += RT) {
    float4 t = Tb[q];
    if (Ub) {
      const float4 u = Ub[q];
      t = make_float4(fmaf(-e, u.x, t.x), fmaf(-e, u.y, t.y), fmaf(-e, u.z, t.z),
                      fmaf(-e, u.w, t.w));
    }
#pragma unroll 4
    for (int i = 0; i < m; i++) {
      const float4 v = Vb[(int64_t)i * Lq + q];
      const float c = sc[i];
      t = make_float4(fmaf(-c, v.x, t.x), fmaf(-c, v.y, t.y), fmaf(-c, v.z, t.z),
                      fmaf(-c, v.w, t.w));
    }
    Tb[q] = t;
    const float w = q < nd4 ? 1.f : 2.f;          // weight of the packed elements
    const float4 tw = make_float4(w * t.x, w * t.y, w * t.z, w * t.w);
    if (norm) {
      nacc = dot4(t, tw, nacc);
    } else {
#pragma unroll 4
      for (int i = 0; i < m; i++)
        sD[i][threadIdx.x] = dot4(Vb[(int64_t)i * Lq + q], tw, sD[i][threadIdx.x]);
    }
  }
  if (norm) {
    const double tot = block_sum((double)nacc, red);
    if (threadIdx.x == 0) partial[(int64_t)b * nchunks + blockIdx.x] = tot;
  } else {
    sd_sums_to_partial(sD, m, partial, b, blockIdx.x, nchunks);
  }
}

__global__ void k32_fix_frozen(int32_t* active, int B) {
  for (int b = threadIdx.x; b < B; b += blockDim.x)
    if (active[b] == 2) active[b] = 0;
}

__global__ void k32_restart_coef(const double* __restrict__ y, double* __restrict__ yp, int m,
                                 int M, const int32_t* __restrict__ active, double* __restrict__ G) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  __shared__ double sy[32], sq[32], sG[32][33];
  const int r = threadIdx.x;
  sy[r] = r < m ? y[(int64_t)b * M + r] : 0.0;
  sq[r] = r < m ? yp[(int64_t)b * M + r] : 0.0;
  for (int i = 0; i < m; i++)
    if (r < m) sG[i][r] = G[(int64_t)b * M * M + (int64_t)i * M + r];
  __syncwarp();
  auto wsum = [](double v) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
  };
  for (int pass = 0; pass < 2; pass++) {
    const double d = wsum(sy[r] * sq[r]);
    sq[r] -= d * sy[r];
    __syncwarp();
  }
  double nq = sqrt(wsum(sq[r] * sq[r]));
  if (!(nq > 1e-14)) {
    double a = r < m ? fabs(sy[r]) : 1e300;
    int idx = r;
    for (int off = 16; off; off >>= 1) {
      const double oa = __shfl_xor_sync(0xffffffffu, a, off);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
      if (oa < a || (oa == a && oi < idx)) { a = oa; idx = oi; }
    }
    sq[r] = (r == idx) ? 1.0 : 0.0;
    __syncwarp();
    const double d = wsum(sy[r] * sq[r]);
    sq[r] -= d * sy[r];
    __syncwarp();
    nq = sqrt(wsum(sq[r] * sq[r]));
  }
  sq[r] /= nq;
  __syncwarp();
  double gy = 0.0, gq = 0.0;
  if (r < m)
    for (int j = 0; j < m; j++) {
      gy = fma(sG[r][j], sy[j], gy);
      gq = fma(sG[r][j], sq[j], gq);
    }
  const double g00 = wsum(sy[r] * gy), g01 = wsum(sy[r] * gq), g11 = wsum(sq[r] * gq);
  const double g10 = wsum(sq[r] * gy);
  if (r < m) yp[(int64_t)b * M + r] = sq[r];
  if (r == 0) {
    double* Gb = G + (int64_t)b * M * M;
    const double off = 0.5 * (g01 + g10);
    Gb[0] = g00;
    Gb[1] = off;
    Gb[M] = off;
    Gb[M + 1] = g11;
  }
}

__global__ void k32_restart_vec(float* __restrict__ V, float* __restrict__ AV, int m, int M,
                                int64_t N, const double* __restrict__ y,
                                const double* __restrict__ q, const int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ float sy[32], sq[32];
  if (threadIdx.x < m) {
    sy[threadIdx.x] = (float)y[(int64_t)b * M + threadIdx.x];
    sq[threadIdx.x] = (float)q[(int64_t)b * M + threadIdx.x];
  }
  __syncthreads();
  float* Vb = V + (int64_t)b * M * N;
  float* AVb = AV + (int64_t)b * M * N;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    float x = 0.f, xp = 0.f, ax = 0.f, axp = 0.f;
    for (int i = 0; i < m; i++) {
      const float v = Vb[(int64_t)i * N + k], av = AVb[(int64_t)i * N + k];
      x = fmaf(sy[i], v, x);
      xp = fmaf(sq[i], v, xp);
      ax = fmaf(sy[i], av, ax);
      axp = fmaf(sq[i], av, axp);
    }
    Vb[k] = x;
    Vb[N + k] = xp;
    AVb[k] = ax;
    AVb[N + k] = axp;
  }
}

__global__ void k32_save_yprev(const double* __restrict__ y, int m, int M, int restarted,
                               const int32_t* __restrict__ active, double* __restrict__ yp) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  for (int i = threadIdx.x; i < M; i += blockDim.x)
    yp[(int64_t)b * M + i] =
        restarted ? (i == 0 ? 1.0 : 0.0) : (i < m ? y[(int64_t)b * M + i] : 0.0);
}

// Diagonal of H + shift S^2 in FP32 for the preconditioner (FP64 where it
// accumulates over a string): e(I) = sum_{p in I} h_pp + 1/2 sum_{p,q in I}
// (J_pq - K_pq) per string, then
//   H_II = e(a) + e(b) + sum_{p in a, q in b} J_pq + shift (nsig - |a & b|)
// with the alpha-beta Coulomb sum taken over pairs p >= q of a | b in a
// fixed order, so that H(a,b) = H(b,a) bitwise.
__global__ void k32_string_energy(const uint32_t* __restrict__ masks, int nstr, int n,
                                  const double* __restrict__ heff_all,
                                  const double* __restrict__ jk_all, float* __restrict__ estr) {
  const int b = blockIdx.y;
  const double* heff = heff_all + (int64_t)b * n * n;
  const double* J = jk_all + (int64_t)b * 2 * n * n;
  const double* K = J + n * n;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nstr; I += gridDim.x * blockDim.x) {
    const uint32_t m = masks[I];
    double e = 0.0, e2 = 0.0;
    for (uint32_t mp = m; mp; mp &= mp - 1) {
      const int p = __ffs(mp) - 1;
      e += heff[p * n + p];
      for (uint32_t mq = m; mq; mq &= mq - 1) {
        const int q = __ffs(mq) - 1;
        e2 += J[p * n + q] - K[p * n + q];
      }
    }
    estr[(int64_t)b * nstr + I] = (float)(e + 0.5 * e2);
  }
}

__global__ void k32_hdiag(const uint32_t* __restrict__ masks, int nstr, int64_t ld, int n,
                          int nsig, const double* __restrict__ jk_all,
                          const float* __restrict__ estr, float shift, float* __restrict__ hd_all) {
  const int b = blockIdx.y;
  __shared__ float sJ[MBE_MAX_ACT * MBE_MAX_ACT];
  for (int t = threadIdx.x; t < n * n; t += blockDim.x)
    sJ[t] = (float)jk_all[(int64_t)b * 2 * n * n + t];
  __syncthreads();
  const int64_t N = (int64_t)nstr * nstr;
  const float* eb = estr + (int64_t)b * nstr;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ia = (int)(i / nstr), ib = (int)(i - (int64_t)ia * nstr);
    if (ia > ib) continue;                      // packed: the upper triangle
    const uint32_t ma = masks[ia], mb = masks[ib], mu = ma | mb;
    float cross = 0.f;
    for (uint32_t mp = mu; mp; mp &= mp - 1) {
      const int p = __ffs(mp) - 1;
      const int ap = (ma >> p) & 1, bp = (mb >> p) & 1;
      for (uint32_t mq = mu & ((2u << p) - 1u); mq; mq &= mq - 1) {
        const int q = __ffs(mq) - 1;
        const int w = q == p ? (ap & bp) : ap * ((mb >> q) & 1) + ((ma >> q) & 1) * bp;
        if (w) cross = fmaf((float)w, sJ[p * n + q], cross);
      }
    }
    hd_all[(int64_t)b * ld + sym_index(ia, ib, nstr)] =
        (eb[ia] + eb[ib]) + cross + shift * (float)(nsig - __popc(ma & mb));
  }
}

__global__ void k32_guess(const float* __restrict__ hd, int nstr, int64_t ld, int M,
                          float* __restrict__ V) {
  const int b = blockIdx.x;
  const int64_t N = (int64_t)nstr * nstr;
  __shared__ float sv[256];
  __shared__ int64_t si[256];
  float best = 3.4e38f;
  int64_t bi = 0;
  for (int64_t k = threadIdx.x; k < N; k += blockDim.x) {
    const int ia = (int)(k / nstr), ib = (int)(k - (int64_t)ia * nstr);
    if (ia > ib) continue;   // the mirror element has the same value, a larger k
    const float v = hd[(int64_t)b * ld + sym_index(ia, ib, nstr)];
    if (v < best) { best = v; bi = k; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) {
      const float o = sv[threadIdx.x + s];
      const int64_t oi = si[threadIdx.x + s];
      if (o < sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  float* Vb = V + (int64_t)b * M * ld;
  for (int64_t k = threadIdx.x; k < ld; k += blockDim.x) Vb[k] = 0.f;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int64_t i0 = si[0];
    const int ia = (int)(i0 / nstr), ib = (int)(i0 % nstr);
    // (|a b> + |b a>) / sqrt(2): its packed element carries both halves
    Vb[sym_index(ia, ib, nstr)] = ia == ib ? 1.f : 0.70710678f;
  }
}

// V0 = X / |X|: packed into V (slot 0), full into F (FP32, input of the
// exact sigma) and C64 (its FP64 copy); Lf is the stride of the full vectors
__global__ void k32_exact_prep(const float* __restrict__ X, const double* __restrict__ xx,
                               float* __restrict__ V, int M, int64_t L, float* __restrict__ F,
                               double* __restrict__ C64, int64_t Lf, int nstr,
                               const int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ float s_inv;
  if (threadIdx.x == 0) s_inv = (float)(1.0 / sqrt(xx[b]));   // one FP64 root per block
  __syncthreads();
  const float inv = s_inv;
  const int64_t N = (int64_t)nstr * nstr;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int ia = (int)(k / nstr), ib = (int)(k - (int64_t)ia * nstr);
    const int64_t p = sym_index(ia, ib, nstr);
    const float v = X[(int64_t)b * L + p] * inv;
    F[(int64_t)b * Lf + k] = v;
    C64[(int64_t)b * Lf + k] = (double)v;
    if (ia <= ib) V[(int64_t)b * M * L + p] = v;
  }
}

// start vectors of the tuples in plan_mask: the full FP32 vectors F (stride
// Lf) written by the parent guess, packed into V (slot 0)
__global__ void k32_pack_start(const float* __restrict__ F, int64_t Lf,
                               const int32_t* __restrict__ plan_mask, int nstr, int M, int64_t L,
                               float* __restrict__ V) {
  const int b = blockIdx.y;
  if (!plan_mask[b]) return;
  const int64_t N = (int64_t)nstr * nstr;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int ia = (int)(k / nstr), ib = (int)(k - (int64_t)ia * nstr);
    if (ia <= ib) V[(int64_t)b * M * L + sym_index(ia, ib, nstr)] = F[(int64_t)b * Lf + k];
  }
}

// partial sums of V0 . A V0 in FP64 (one FP64 FMA per element)
__global__ void k32_exact_xax(const double* __restrict__ C64, const double* __restrict__ S64,
                              int64_t N, int ch, int nchunks, const int32_t* __restrict__ active,
                              double* __restrict__ partial) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double red[32];
  const int64_t k0 = (int64_t)blockIdx.x * ch, k1 = min(N, k0 + ch);
  double acc = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x)
    acc = fma(C64[(int64_t)b * N + k], S64[(int64_t)b * N + k], acc);
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) partial[(int64_t)b * nchunks + blockIdx.x] = tot;
}

// r_x = A V0 - theta_x V0 (stored FP32) and partial sums of |r_x|^2
// (C64, S64 full, stride N; RX packed, stride L)
__global__ void k32_exact_rx(const double* __restrict__ C64, const double* __restrict__ S64,
                             const double* __restrict__ thx, int64_t N, int ch, int nchunks,
                             const int32_t* __restrict__ active, float* __restrict__ RX,
                             int64_t L, int nstr, double* __restrict__ partial) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double red[32];
  const double th = thx[b];
  const int64_t k0 = (int64_t)blockIdx.x * ch, k1 = min(N, k0 + ch);
  double acc = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double r = fma(-th, C64[(int64_t)b * N + k], S64[(int64_t)b * N + k]);
    const int ia = (int)(k / nstr), ib = (int)(k - (int64_t)ia * nstr);
    if (ia <= ib && ia < nstr) RX[(int64_t)b * L + sym_index(ia, ib, nstr)] = (float)r;
    acc = fma(r, r, acc);
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) partial[(int64_t)b * nchunks + blockIdx.x] = tot;
}

// theta_x = xAx / xx; G = [[xAx]]; rnorm from the partials; y = [1]
__global__ void k32_exact_fin(const double* __restrict__ xax, const double* __restrict__ xx,
                              const double* __restrict__ rpart, int nchunks, int M, int B,
                              const int32_t* __restrict__ active, double* __restrict__ thx,
                              double* __restrict__ theta, double* __restrict__ G,
                              double* __restrict__ rnorm, int32_t* __restrict__ iters) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    if (!active[b]) continue;
    const double t = xax[b] / xx[b];
    thx[b] = t;
    theta[b] = t;
    G[(int64_t)b * M * M] = xax[b];
    double s = 0.0;
    for (int c = 0; c < nchunks; c++) s += rpart[(int64_t)b * nchunks + c];
    rnorm[b] = sqrt(s);
    iters[b] += 1;
  }
}

// target of tuple b: max(abs_target, rel_target max(1, |theta_x|)); the FP32
// storage of x puts a floor of a few 1e-8 |A| on its exact residual
// rnorm of the tuples in `mask` arrives as |r_x|^2 and leaves as |r_x|
__global__ void k32_select(double* __restrict__ rnorm, const int32_t* __restrict__ mask,
                           const double* __restrict__ thx, int B, double abs_target,
                           double rel_target, double drop, int32_t* __restrict__ active,
                           double* __restrict__ tolr, int32_t* __restrict__ nactive) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double target = fmax(abs_target, rel_target * fmax(1.0, fabs(thx[b])));
    double r = rnorm[b];
    if (mask[b]) {
      r = sqrt(fmax(0.0, r));
      rnorm[b] = r;
    }
    const int a = (mask[b] && r > target) ? 1 : 0;
    active[b] = a;
    tolr[b] = fmax(target, drop * r);
    if (a) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *nactive = cnt;
}

__global__ void k32_fill_i(int32_t* v, int n, int32_t x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = x;
}
__global__ void k32_fill_d(double* v, int n, double x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = x;
}
__global__ void k32_copy_i(const int32_t* s, int32_t* d, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

}  // namespace

void davidson_batch_mixed(mbe_ctx* ctx, BinProblem& bp, double* e_out_host, int32_t* status_host,
                          double* x_out_dev, const GuessPlan* plan) {
  const int B = bp.B;
  // Ms: the subspace cap of the first stage and of a refinement round; M: the
  // allocated size (stride), the cap of the rounds after one that ended with
  // its subspace full and tuples still above their targets
  const int Ms = std::max(4, std::min(32, ctx->opt.max_subspace));
  const int M = mixed_subspace_alloc(ctx->opt.max_subspace);
  // N determinants per tuple; every FP32 Davidson vector is packed (L =
  // sym_len elements), the FP64 exact-point vectors and the FP32 input of the
  // exact sigma are full (Lf = N rounded up to a multiple of 4).  Padding
  // stays zero: no kernel writes it, and every combination of zero elements
  // is zero.
  const int64_t N = bp.ndet, L = sym_len(bp.nstr), Lf = (N + 3) / 4 * 4;
  const int64_t nd4 = sym_nd(bp.nstr) / 4;
  const double shift = ctx->opt.spin_shift;
  DevPool* P = &ctx->pool;
  const int nsm = [&] {
    int v = 0;
    CU_CHECK(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device));
    return v;
  }();
  // reduction chunk: about four CTAs per SM over the batch, 1024..16384
  // elements (a multiple of 1024)
  int ch = 16384;
  while (ch > 1024 && (int64_t)B * ((L + ch - 1) / ch) < 4 * (int64_t)nsm) ch >>= 1;
  const int nchunks = (int)((L + ch - 1) / ch);
  const int nchunks_f = (int)((Lf + ch - 1) / ch);   // chunks of the full FP64 vectors
  DevBuf<float> V(P, (size_t)B * M * L), AV(P, (size_t)B * M * L), hd(P, (size_t)B * L),
      T(P, (size_t)B * L), X(P, (size_t)B * L), RX(P, (size_t)B * L), F(P, (size_t)B * Lf);
  DevBuf<double> C64(P, (size_t)B * Lf), S64(P, (size_t)B * Lf),
      G(P, (size_t)B * M * M), y(P, (size_t)B * M), yp(P, (size_t)B * M), theta(P, B),
      thx(P, B), rnorm(P, B), tolr(P, B), coef(P, (size_t)B * M), cdot(P, B), rdot(P, B),
      xx(P, B), xax(P, B), partial(P, (size_t)B * M * nchunks),
      rpart(P, (size_t)B * std::max(nchunks, nchunks_f));
  DevBuf<int32_t> active(P, B), iters(P, B), nact(P, 1), mask(P, B);
  SigmaWork sw;
  cudaStream_t st = ctx->stream;
  // zero padding (the vectors' tails are read by the streaming kernels)
  CU_CHECK(cudaMemsetAsync(V.ptr, 0, sizeof(float) * B * M * L, st));
  CU_CHECK(cudaMemsetAsync(AV.ptr, 0, sizeof(float) * B * M * L, st));
  CU_CHECK(cudaMemsetAsync(hd.ptr, 0, sizeof(float) * B * L, st));
  CU_CHECK(cudaMemsetAsync(RX.ptr, 0, sizeof(float) * B * L, st));
  if (Lf != N) {
    CU_CHECK(cudaMemsetAsync(F.ptr, 0, sizeof(float) * B * Lf, st));
    CU_CHECK(cudaMemsetAsync(C64.ptr, 0, sizeof(double) * B * Lf, st));
    CU_CHECK(cudaMemsetAsync(S64.ptr, 0, sizeof(double) * B * Lf, st));
  }
  const int64_t eb = std::min<int64_t>((L + 255) / 256, 1024);
  const int64_t ebf = std::min<int64_t>((Lf + 255) / 256, 1024);
  const dim3 ge((unsigned)eb, B), gef((unsigned)ebf, B), gc(nchunks, B), gcf(nchunks_f, B);
  const int max_iter = std::max(1, ctx->opt.max_iter);
  int total_it = 0;
  int64_t vecs_tc = 0, vecs_ex = 0;

  // diagonal (FP64 kernel shared with the FP64 mode), kept in FP32
  {
    DevBuf<float> estr(P, (size_t)B * bp.nstr);
    k32_string_energy<<<dim3((unsigned)((bp.nstr + 255) / 256), B), 256, 0, st>>>(
        bp.tab->masks.ptr, bp.nstr, bp.n, bp.heff.ptr, bp.jk.ptr, estr.ptr);
    CU_LAUNCH_CHECK();
    k32_hdiag<<<gef, 256, 0, st>>>(bp.tab->masks.ptr, bp.nstr, L, bp.n, bp.nsig, bp.jk.ptr,
                                  estr.ptr, (float)shift, hd.ptr);
    CU_LAUNCH_CHECK();
  }
  // P-space preconditioner: the lowest-diagonal block of A solved exactly,
  // with Olsen's correction (u = M^-1 x in U32, its dot partials in upart,
  // x.M^-1 r and x.M^-1 x in xpart)
  PspaceWork psp;
  pspace_setup(ctx, bp, hd.ptr, L, shift, pspace_size(bp, ctx->opt.pspace), psp);
  const bool olsen = psp.npp > 0;
  DevBuf<float> U32(P, olsen ? (size_t)B * L : 0), epsb(P, olsen ? (size_t)B : 0);
  DevBuf<double> upart(P, olsen ? (size_t)B * M * nchunks : 0),
      xpart(P, olsen ? (size_t)B * 2 * nchunks : 0), xsum(P, olsen ? (size_t)B * 2 : 0),
      coef2(P, olsen ? (size_t)B * M : 0);
  {
    // the residual kernel's dot accumulators: up to 2 x 32 x RT floats
    static bool attr_done[MBE_MAX_DEVICES] = {false};
    once_per_device(attr_done, ctx->device, [] {
      CU_CHECK(cudaFuncSetAttribute(k32_residual_pre, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    2 * 32 * RT * (int)sizeof(float)));
    });
  }
  k32_guess<<<B, 256, 0, st>>>(hd.ptr, bp.nstr, L, M, V.ptr);
  CU_LAUNCH_CHECK();
  if (plan) {
    // the parent guess writes full vectors (into F), packed into V_0 here
    launch_parent_guess(ctx, *plan, bp.n, bp.nsig, bp.nstr, F.ptr, nullptr, Lf);
    std::vector<int32_t> pm(B, 0);
    for (int b : plan->b) pm[b] = 1;
    DevBuf<int32_t> pmask(P, B);
    CU_CHECK(cudaMemcpyAsync(pmask.ptr, pm.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, st));
    k32_pack_start<<<gef, 256, 0, st>>>(F.ptr, Lf, pmask.ptr, bp.nstr, M, L, V.ptr);
    CU_LAUNCH_CHECK();
    CU_CHECK(cudaStreamSynchronize(st));   // pm is read by the copy above
  }
  k32_fill_i<<<1, 256, 0, st>>>(active.ptr, B, 1);
  CU_LAUNCH_CHECK();
  CU_CHECK(cudaMemsetAsync(iters.ptr, 0, sizeof(int32_t) * B, st));
  CU_CHECK(cudaMemsetAsync(G.ptr, 0, sizeof(double) * B * M * M, st));
  k32_fill_d<<<1, 256, 0, st>>>(tolr.ptr, B, ctx->opt.mixed_stage_tol);
  CU_LAUNCH_CHECK();

  auto dots = [&](const float* Xv, int64_t xb, int64_t xv, const float* Yv, int64_t yb, int m,
                  double* out, int64_t ob, int64_t oi, const int32_t* act) {
    k32_multidot<<<dim3(nchunks, B), RT, 0, st>>>(Xv, xb, xv, Yv, yb, m, L, nd4, ch, nchunks,
                                                   act, partial.ptr);
    CU_LAUNCH_CHECK();
    k32_final<<<B, 32, 0, st>>>(partial.ptr, m, nchunks, act, out, ob, oi);
    CU_LAUNCH_CHECK();
  };
  auto dot_comp = [&](const float* Xv, int64_t xb, const float* Yv, int64_t yb, double* out,
                      const int32_t* act) {
    k32_dot_comp<<<dim3(nchunks, B), RT, 0, st>>>(Xv, xb, Yv, yb, L, 4 * nd4, ch, nchunks, act,
                                                   partial.ptr);
    CU_LAUNCH_CHECK();
    k32_final<<<B, 32, 0, st>>>(partial.ptr, 1, nchunks, act, out, 1, 1);
    CU_LAUNCH_CHECK();
  };
  auto count_active = [&]() {
    int32_t n = 0;
    CU_CHECK(cudaMemcpyAsync(&n, nact.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CU_CHECK(cudaStreamSynchronize(st));
    if (ctx->opt.verbose) {
      std::vector<double> rn(B), th(B);
      CU_CHECK(cudaMemcpy(rn.data(), rnorm.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost));
      CU_CHECK(cudaMemcpy(th.data(), theta.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost));
      double mx = 0.0;
      for (double r : rn) mx = std::max(mx, r);
      fprintf(stderr, "[mbe mixed] n=%d nsig=%d B=%d it=%d active=%d max|r|=%.3e theta0=%.12f\n",
              bp.n, bp.nsig, B, total_it, n, mx, th[0]);
    }
    return n;
  };
  // orthogonalise T against V[0..m) twice (classical Gram-Schmidt), append
  // as V[m].  raw: T is an unpreconditioned residual; dots_ready: T is
  // preconditioned and `partial` holds the first pass's V_i . T partials
  // (both from k32_residual_pre).  The P-space block of the correction is
  // replaced first (the dot partials corrected with it).
  auto extend = [&](int m, bool raw, bool dots_ready) {
    if (raw) {
      k32_precondition<<<ge, 256, 0, st>>>(T.ptr, hd.ptr, L, theta.ptr, active.ptr);
      CU_LAUNCH_CHECK();
    }
    // Olsen's combination goes with the P-space block (its exact block would
    // return t = -x); the exact-point residual (raw) takes the plain block
    const bool ols = olsen && !raw;
    pspace_apply(ctx, bp, psp, T.ptr, hd.ptr, L, theta.ptr, V.ptr, m, M, nchunks, partial.ptr,
                 dots_ready, active.ptr, ols, U32.ptr, X.ptr, upart.ptr, xpart.ptr);
    if (ols) {
      k32_final<<<B, 32, 0, st>>>(xpart.ptr, 2, nchunks, active.ptr, xsum.ptr, 2, 1);
      CU_LAUNCH_CHECK();
      if (dots_ready) {
        k32_final<<<B, 32, 0, st>>>(partial.ptr, m, nchunks, active.ptr, coef.ptr, M, 1);
        CU_LAUNCH_CHECK();
        k32_final<<<B, 32, 0, st>>>(upart.ptr, m, nchunks, active.ptr, coef2.ptr, M, 1);
        CU_LAUNCH_CHECK();
      }
      k32_olsen<<<B, 32, 0, st>>>(xsum.ptr, coef2.ptr, m, M, dots_ready ? 1 : 0, active.ptr,
                                  coef.ptr, epsb.ptr);
      CU_LAUNCH_CHECK();
      if (!dots_ready) {
        k32_sub_eps<<<ge, 256, 0, st>>>(T.ptr, U32.ptr, epsb.ptr, L, active.ptr);
        CU_LAUNCH_CHECK();
        dots(V.ptr, (int64_t)M * L, L, T.ptr, L, m, coef.ptr, M, 1, active.ptr);
      }
    } else if (dots_ready) {
      k32_final<<<B, 32, 0, st>>>(partial.ptr, m, nchunks, active.ptr, coef.ptr, M, 1);
      CU_LAUNCH_CHECK();
    } else {
      dots(V.ptr, (int64_t)M * L, L, T.ptr, L, m, coef.ptr, M, 1, active.ptr);
    }
    for (int pass = 0; pass < 2; pass++) {
      const bool fold = ols && dots_ready && pass == 0;   // t = t1 - eps u inside the pass
      k32_orth_pass<<<gc, RT, 0, st>>>(T.ptr, V.ptr, m, M, L, nd4, coef.ptr, active.ptr, pass, ch,
                                      nchunks, partial.ptr, fold ? U32.ptr : nullptr,
                                      epsb.ptr);
      CU_LAUNCH_CHECK();
      k32_final<<<B, 32, 0, st>>>(partial.ptr, pass ? 1 : m, nchunks, active.ptr, coef.ptr, M,
                                  1);
      CU_LAUNCH_CHECK();
    }
    k32_append<<<ge, 256, 0, st>>>(T.ptr, V.ptr, m, M, L, coef.ptr, active.ptr);
    CU_LAUNCH_CHECK();
    k32_fix_frozen<<<1, 256, 0, st>>>(active.ptr, B);
    CU_LAUNCH_CHECK();
  };
  // Davidson iterations from a subspace of m_start vectors, the newest one's
  // sigma pending; exact0: V_0 is an exact point (no restart: the stage ends
  // when the subspace is full)
  // returns true when an exact0 stage ended because its subspace (mcap
  // vectors) was full with tuples still iterating
  //
  // An iteration is a head (sigma vector of V[m-1], subspace row, Ritz
  // step, residual and correction, convergence flags), one synchronisation
  // (the number of tuples still iterating), then a tail (restart when the
  // subspace is full, the next vector V[m]).  The tail is issued together
  // with the next head, so that with opt.graphs one CUDA graph per
  // iteration carries both: the host makes one launch and one
  // synchronisation per iteration.  The graph's shape depends only on
  // (exact0, tail present, restart); m changes pointers and loop bounds,
  // which the in-place update of the executable graph takes.
  // (the legacy default stream cannot be captured: plain launches there)
  const bool use_graphs = ctx->opt.graphs != 0 && st != nullptr && st != cudaStreamLegacy;
  GraphRunner gr(st);
  auto tail = [&](int m_full, bool restart) {
    int m = m_full;
    if (restart) {
      k32_restart_coef<<<B, 32, 0, st>>>(y.ptr, yp.ptr, m, M, active.ptr, G.ptr);
      CU_LAUNCH_CHECK();
      k32_restart_vec<<<ge, 256, 0, st>>>(V.ptr, AV.ptr, m, M, L, y.ptr, yp.ptr, active.ptr);
      CU_LAUNCH_CHECK();
      m = 2;
    }
    k32_save_yprev<<<B, 32, 0, st>>>(y.ptr, m, M, restart ? 1 : 0, active.ptr, yp.ptr);
    CU_LAUNCH_CHECK();
    // after a restart V changed: the first pass's dots are taken again
    extend(m, false, !restart);
  };
  auto head = [&](int m, int it, int m_start, int rel, bool exact0) {
    sigma_tc(ctx, bp, sw, V.ptr + (int64_t)(m - 1) * L, (int64_t)M * L,
             AV.ptr + (int64_t)(m - 1) * L, (int64_t)M * L, active.ptr, shift, true);
    dots(V.ptr, (int64_t)M * L, L, AV.ptr + (int64_t)(m - 1) * L, (int64_t)M * L, m, coef.ptr,
         M, 1, active.ptr);
    if (exact0) {
      dot_comp(V.ptr, (int64_t)M * L, V.ptr + (int64_t)(m - 1) * L, (int64_t)M * L, cdot.ptr,
               active.ptr);
      dots(RX.ptr, L, 0, V.ptr + (int64_t)(m - 1) * L, (int64_t)M * L, 1, rdot.ptr, 1, 1,
           active.ptr);
    }
    k32_store_row<<<B, 32, 0, st>>>(coef.ptr, cdot.ptr, rdot.ptr, thx.ptr, m, M, exact0 ? 1 : 0,
                                    active.ptr, G.ptr);
    CU_LAUNCH_CHECK();
    k32_jacobi<<<B, 32, 0, st>>>(G.ptr, m, M, active.ptr, theta.ptr, y.ptr);
    CU_LAUNCH_CHECK();
    k32_residual_pre<<<gc, RT, (olsen ? 2 : 1) * m * RT * sizeof(float), st>>>(
        V.ptr, AV.ptr, RX.ptr, exact0 ? 1 : 0, m, M, L, nd4, y.ptr, theta.ptr, thx.ptr, hd.ptr,
        active.ptr, X.ptr, T.ptr, ch, nchunks, rpart.ptr, partial.ptr, olsen ? 1 : 0, U32.ptr,
        upart.ptr, xpart.ptr);
    CU_LAUNCH_CHECK();
    k32_converge<<<1, 256, 0, st>>>(rpart.ptr, nchunks, B, m_start > 1 ? it + 1 : it, tolr.ptr,
                                    rel, theta.ptr, rnorm.ptr, active.ptr, iters.ptr, nact.ptr);
    CU_LAUNCH_CHECK();
  };
  // round_start: a refinement round's first correction (the preconditioned
  // exact residual, appended as V_1) goes with the round's first head
  auto round_start = [&] {
    k32_copy_i<<<1, 256, 0, st>>>(active.ptr, mask.ptr, B);
    CU_LAUNCH_CHECK();
    CU_CHECK(cudaMemcpyAsync(T.ptr, RX.ptr, sizeof(float) * B * L, cudaMemcpyDeviceToDevice, st));
    k32_save_yprev<<<B, 32, 0, st>>>(y.ptr, 1, M, 1, active.ptr, yp.ptr);
    CU_LAUNCH_CHECK();
    extend(1, true, false);
  };
  auto stage = [&](int m_start, int cap, int rel, bool exact0, int nact0, int mcap) -> bool {
    int m = m_start, nact_h = nact0;
    bool pending = false, restart = false;   // the tail still to issue
    int m_tail = 0;
    if (exact0 && (cap <= 0 || total_it >= max_iter)) round_start();
    for (int it = 0; it < cap && total_it < max_iter; it++, total_it++) {
      const bool pend = pending, rs = restart, pro = exact0 && it == 0;
      const int mt = m_tail;
      auto body = [&] {
        if (pro) round_start();
        if (pend) tail(mt, rs);
        head(m, it, m_start, rel, exact0);
      };
      // the first iteration of a batch runs as plain launches: it makes the
      // one-time set-up of the sigma path (tables, operand plans, the
      // autotuner's timed launches), which synchronises
      if (use_graphs && total_it >= 1)
        gr.run((exact0 ? 1 : 0) | (pend ? 2 : 0) | (pend && rs ? 4 : 0) | (pro ? 8 : 0), body);
      else
        body();
      pending = false;
      vecs_tc += nact_h;
      nact_h = count_active();
      if (nact_h == 0) return false;
      if (exact0 && m == mcap) return true;
      restart = m == mcap;
      m_tail = m;
      pending = true;
      m = (restart ? 2 : m) + 1;
    }
    if (pending) tail(m_tail, restart);
    return false;
  };
  // the exact-point sigma: fused on the tensor cores where it fits (kpad <= 80)
  const bool exact_fused = sigma_exact_supported(bp.npair, bp.nstr);
  // exact point of the tuples in `mask`: V0 = x/|x|, exact A V0, theta_x,
  // r_x and its norm; G = [[V0.AV0]]
  auto exact_point = [&]() {
    k32_copy_i<<<1, 256, 0, st>>>(mask.ptr, active.ptr, B);
    CU_LAUNCH_CHECK();
    dot_comp(X.ptr, L, X.ptr, L, xx.ptr, active.ptr);
    k32_exact_prep<<<gef, 256, 0, st>>>(X.ptr, xx.ptr, V.ptr, M, L, F.ptr, C64.ptr, Lf, bp.nstr,
                                        active.ptr);
    CU_LAUNCH_CHECK();
    dot_comp(V.ptr, (int64_t)M * L, V.ptr, (int64_t)M * L, xx.ptr, active.ptr);
    if (exact_fused) {
      sigma_exact(ctx, bp, sw, F.ptr, Lf, S64.ptr, Lf, active.ptr);
      launch_finish_sym_fp64(ctx, bp, S64.ptr, Lf, C64.ptr, Lf, shift, active.ptr);
    } else {
      sigma_fp64(ctx, bp, sw, C64.ptr, Lf, S64.ptr, Lf, active.ptr, shift, true, true);
    }
    vecs_ex += B;
    k32_exact_xax<<<gcf, RT, 0, st>>>(C64.ptr, S64.ptr, Lf, ch, nchunks_f, active.ptr,
                                      rpart.ptr);
    CU_LAUNCH_CHECK();
    k32_final<<<B, 32, 0, st>>>(rpart.ptr, 1, nchunks_f, active.ptr, xax.ptr, 1, 1);
    CU_LAUNCH_CHECK();
    // theta_x first (the residual needs it), then r_x and its norm
    k32_exact_fin<<<(B + 127) / 128, 128, 0, st>>>(xax.ptr, xx.ptr, rpart.ptr, 0, M, B,
                                                   active.ptr, thx.ptr, theta.ptr, G.ptr,
                                                   rnorm.ptr, iters.ptr);
    CU_LAUNCH_CHECK();
    k32_exact_rx<<<gcf, RT, 0, st>>>(C64.ptr, S64.ptr, thx.ptr, Lf, ch, nchunks_f, active.ptr,
                                     RX.ptr, L, bp.nstr, rpart.ptr);
    CU_LAUNCH_CHECK();
    k32_final<<<B, 32, 0, st>>>(rpart.ptr, 1, nchunks_f, active.ptr, rnorm.ptr, 1, 1);
    CU_LAUNCH_CHECK();
  };

  // the exact path's set-up before any of its calls is captured
  if (exact_fused) sigma_exact_prepare(ctx, bp, sw);
  // stage A
  stage(1, 150, 1, false, B, Ms);
  // refinement rounds
  const double abs_target = ctx->opt.conv_tol_r, rel_target = ctx->opt.mixed_rel_tol;
  k32_fill_i<<<1, 256, 0, st>>>(mask.ptr, B, 1);
  CU_LAUNCH_CHECK();
  int round_cap = Ms;
  for (int round = 0; round < 12; round++) {
    // the exact point and the selection of the tuples above their targets
    // (one graph; the unfused FP64 path stages host data and runs plain)
    auto point = [&] {
      exact_point();
      k32_select<<<1, 256, 0, st>>>(rnorm.ptr, mask.ptr, thx.ptr, B, abs_target, rel_target,
                                    ctx->opt.mixed_round_drop, active.ptr, tolr.ptr, nact.ptr);
      CU_LAUNCH_CHECK();
    };
    if (use_graphs && exact_fused)
      gr.run(16, point);
    else
      point();
    const int na = count_active();
    if (ctx->opt.verbose) {
      double t0 = 0.0, r0 = 0.0;
      CU_CHECK(cudaMemcpy(&t0, thx.ptr, sizeof(double), cudaMemcpyDeviceToHost));
      CU_CHECK(cudaMemcpy(&r0, rnorm.ptr, sizeof(double), cudaMemcpyDeviceToHost));
      fprintf(stderr, "[mbe mixed] exact point %d: %d above target; theta_x0=%.15f |r_x0|=%.3e\n",
              round, na, t0, r0);
    }
    if (na == 0 || total_it >= max_iter) break;
    // the exact residual, preconditioned, is the first correction: issued
    // with the round's first iteration (round_start)
    // a round that filled its subspace before its tuples reached the target
    // (near-degenerate spaces) makes the later rounds use all M vectors
    if (stage(2, 40, 0, true, na, round_cap)) round_cap = M;
  }
  if (sigma_tc_error(ctx, sw)) throw MbeError{MBE_ETIMEOUT, "tensor-core sigma wait timed out"};

  // energies: E = E_core + theta_x - shift <S^2> (S^2 of the exact-point vector, FP64)
  s2_apply(ctx, bp, C64.ptr, Lf, S64.ptr, Lf, nullptr);
  std::vector<double> th(B), ec(B), rn(B), s2(B), nx(B);
  std::vector<int32_t> it_h(B);
  {
    // <S^2> = C64.S64 / C64.C64 via the FP64 partial-sum kernel
    DevBuf<int32_t> all(P, B);
    k32_fill_i<<<1, 256, 0, st>>>(all.ptr, B, 1);
    CU_LAUNCH_CHECK();
    k32_exact_xax<<<gcf, RT, 0, st>>>(C64.ptr, S64.ptr, Lf, ch, nchunks_f, all.ptr, rpart.ptr);
    CU_LAUNCH_CHECK();
    k32_final<<<B, 32, 0, st>>>(rpart.ptr, 1, nchunks_f, all.ptr, coef.ptr, 1, 1);
    CU_LAUNCH_CHECK();
    k32_exact_xax<<<gcf, RT, 0, st>>>(C64.ptr, C64.ptr, Lf, ch, nchunks_f, all.ptr, rpart.ptr);
    CU_LAUNCH_CHECK();
    k32_final<<<B, 32, 0, st>>>(rpart.ptr, 1, nchunks_f, all.ptr, xax.ptr, 1, 1);
    CU_LAUNCH_CHECK();
  }
  CU_CHECK(cudaMemcpyAsync(th.data(), thx.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(ec.data(), bp.ecore.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(rn.data(), rnorm.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(s2.data(), coef.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(nx.data(), xax.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(it_h.data(), iters.ptr, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
  if (x_out_dev)
    CU_CHECK(cudaMemcpy2DAsync(x_out_dev, sizeof(double) * N, C64.ptr, sizeof(double) * Lf,
                               sizeof(double) * N, B, cudaMemcpyDeviceToDevice, st));
  CU_CHECK(cudaStreamSynchronize(st));

  for (int b = 0; b < B; b++) {
    const double s2n = nx[b] > 0.0 ? s2[b] / nx[b] : 0.0;
    if (ctx->opt.verbose)
      fprintf(stderr, "[mbe mixed] tuple %d: theta_x=%.15f <S^2>=%.3e |r_x|=%.3e E_core=%.12f\n", b,
              th[b], s2n, rn[b], ec[b]);
    if (e_out_host) e_out_host[b] = ec[b] + th[b] - shift * s2n;
    const bool ok = rn[b] <= 10.0 * std::max(abs_target, rel_target * std::max(1.0, std::fabs(th[b])));
    if (status_host) status_host[b] = ok ? MBE_OK : MBE_ENOCONV;
    ctx->stats.iters_total += it_h[b];
    ctx->stats.iters_max = std::max<int64_t>(ctx->stats.iters_max, it_h[b]);
    ctx->stats.noconv += ok ? 0 : 1;
  }
  const double per = 2.0 * (double)N * bp.npair * bp.npair;
  ctx->stats.graph_launches += gr.launched;
  ctx->stats.graph_builds += gr.instantiated;
  ctx->stats.casci += B;
  ctx->stats.sigma_vectors += vecs_tc + vecs_ex;
  ctx->stats.sigma_flops += (double)(vecs_tc + vecs_ex) * per;
  ctx->stats.dom_flops += (double)vecs_tc * per;
  ctx->stats.fp64_flops += (double)vecs_ex * per;
}
