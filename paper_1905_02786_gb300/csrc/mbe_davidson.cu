// Batched Davidson iteration (Davidson, J. Comput. Phys. 17, 87 (1975)) for
// the lowest singlet of every CASCI of one bin in the FP64 and emulated-FP64
// modes (the mixed mode's Davidson is in mbe_davidson32.cu), FP64 throughout:
//   K5  batched projections V^T w (two-phase, fixed-order reductions)
//   K6  Rayleigh-Ritz: cyclic Jacobi on the m x m projected matrix, one warp
//       per tuple
//   K7  residual r = AV y - theta V y, diagonal preconditioner
//       t = r / (theta - H_II) with |denominator| >= 1e-8, two-pass
//       Gram-Schmidt, normalisation
// The operator is H_active + spin_shift * S^2 restricted to the alpha<->beta
// symmetric vectors; the start vector is the lowest diagonal determinant,
// symmetrised.  All tuples of a batch share the subspace size m; a tuple
// that has converged is frozen (every kernel skips it).
#include "mbe_internal.cuh"
#include "mbe_ritz.cuh"
#include <algorithm>
#include <cmath>
#include <cstdio>

namespace {

constexpr int DOT_CHUNK = 4096;

// partial[b][i][chunk] = sum over the chunk of X[b][i][k] * y[b][k], i < m
__global__ void k_multidot_partial(const double* __restrict__ X, int64_t x_bstride,
                                   int64_t x_vstride, const double* __restrict__ Y,
                                   int64_t y_bstride, int m, int64_t N, int nchunks,
                                   const int32_t* __restrict__ active, double* __restrict__ partial) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int chunk = blockIdx.x;
  const int64_t k0 = (int64_t)chunk * DOT_CHUNK;
  const int64_t k1 = min(N, k0 + DOT_CHUNK);
  __shared__ double red[32][33];
  const double* yb = Y + (int64_t)b * y_bstride;
  for (int i0 = 0; i0 < m; i0 += 32) {
    double acc[32];
    const int ni = min(32, m - i0);
#pragma unroll
    for (int i = 0; i < 32; i++) acc[i] = 0.0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      double yv = yb[k];
#pragma unroll
      for (int i = 0; i < 32; i++)
        if (i < ni) acc[i] = fma(X[(int64_t)b * x_bstride + (int64_t)(i0 + i) * x_vstride + k], yv, acc[i]);
    }
    // reduce over the block: warp shuffle then shared memory (fixed order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 32; i++) {
      double v = acc[i];
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

__global__ void k_multidot_final(const double* __restrict__ partial, int m, int nchunks,
                                 const int32_t* __restrict__ active, double* __restrict__ out,
                                 int64_t out_bstride, int64_t out_istride) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double* p = partial + ((int64_t)b * m + i) * nchunks;
    double s = 0.0;
    for (int c = 0; c < nchunks; c++) s += p[c];
    out[(int64_t)b * out_bstride + (int64_t)i * out_istride] = s;
  }
}

// G[b][j][i] = G[b][i][j] = dots[b][i] for i < m (row/column j = m-1)
__global__ void k_store_grow(const double* __restrict__ dots, int m, int M,
                             const int32_t* __restrict__ active, double* __restrict__ G) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  const int j = m - 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double v = dots[(int64_t)b * M + i];
    G[(int64_t)b * M * M + (int64_t)j * M + i] = v;
    G[(int64_t)b * M * M + (int64_t)i * M + j] = v;
  }
}

// lowest eigenpair of the m x m subspace matrix G[b] (one warp per tuple)
__global__ void k_jacobi(const double* __restrict__ G, int m, int M,
                        const int32_t* __restrict__ active, double* __restrict__ theta,
                        double* __restrict__ y) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  __shared__ RitzShared S;
  ritz_lowest(G + (int64_t)b * M * M, m, M, S, theta + b, y + (int64_t)b * M);
}

// x = V y, T = AV y - theta x, partial ||T||^2; X receives x.
__global__ void k_residual(const double* __restrict__ V, const double* __restrict__ AV, int m,
                           int M, int64_t N, const double* __restrict__ y,
                           const double* __restrict__ theta, const int32_t* __restrict__ active,
                           double* __restrict__ X, double* __restrict__ T, int nchunks,
                           double* __restrict__ partial) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double sy[32];
  __shared__ double red[32];
  if (threadIdx.x < m) sy[threadIdx.x] = y[(int64_t)b * M + threadIdx.x];
  __syncthreads();
  const double th = theta[b];
  const int64_t k0 = (int64_t)blockIdx.x * DOT_CHUNK, k1 = min(N, k0 + DOT_CHUNK);
  const double* Vb = V + (int64_t)b * M * N;
  const double* AVb = AV + (int64_t)b * M * N;
  double acc = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double x = 0.0, ax = 0.0;
    for (int i = 0; i < m; i++) {
      x = fma(sy[i], Vb[(int64_t)i * N + k], x);
      ax = fma(sy[i], AVb[(int64_t)i * N + k], ax);
    }
    double r = ax - th * x;
    X[(int64_t)b * N + k] = x;
    T[(int64_t)b * N + k] = r;
    acc = fma(r, r, acc);
  }
  for (int off = 16; off; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
    partial[(int64_t)b * nchunks + blockIdx.x] = s;
  }
}

// convergence bookkeeping after the residual norms are known
__global__ void k_converge(const double* __restrict__ partial, int nchunks, int B, int it,
                           const double* __restrict__ tol_r, double tol_e, int rel,
                           const double* __restrict__ theta,
                           double* __restrict__ theta_old, double* __restrict__ rnorm,
                           int32_t* __restrict__ active, int32_t* __restrict__ iters,
                           int32_t* __restrict__ nactive) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (!active[b]) continue;
    double s = 0.0;
    for (int c = 0; c < nchunks; c++) s += partial[(int64_t)b * nchunks + c];
    double rn = sqrt(s);
    rnorm[b] = rn;
    iters[b] += 1;
    // rel: the residual tolerance scales with max(1, |theta|) (the floor of a
    // reduced-precision sigma is relative to the size of H)
    const double tr = rel ? tol_r[b] * fmax(1.0, fabs(theta[b])) : tol_r[b];
    bool conv = it > 0 && fabs(theta[b] - theta_old[b]) < tol_e && rn < tr;
    theta_old[b] = theta[b];
    if (conv) active[b] = 0;
    else atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *nactive = cnt;
}

// Restart keeping two vectors: the current Ritz vector x = V y and the
// previous one, orthonormalised against x in coefficient space
// (q = y_prev - (y.y_prev) y, twice, normalised; V is orthonormal, so this
// avoids the cancellation of subtracting two nearly parallel long vectors).
// The new 2x2 projected matrix is [y q]^T G [y q].  One warp per tuple.
__global__ void k_restart_coef(const double* __restrict__ y, double* __restrict__ yp, int m, int M,
                               const int32_t* __restrict__ active, double* __restrict__ G) {
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
    double d = wsum(sy[r] * sq[r]);
    sq[r] -= d * sy[r];
    __syncwarp();
  }
  double nq = sqrt(wsum(sq[r] * sq[r]));
  if (!(nq > 1e-14)) {
    // x did not move: take the unit vector on which x has least weight
    double a = r < m ? fabs(sy[r]) : 1e300;
    int idx = r;
    for (int off = 16; off; off >>= 1) {
      double oa = __shfl_xor_sync(0xffffffffu, a, off);
      int oi = __shfl_xor_sync(0xffffffffu, idx, off);
      if (oa < a || (oa == a && oi < idx)) { a = oa; idx = oi; }
    }
    sq[r] = (r == idx) ? 1.0 : 0.0;
    __syncwarp();
    double d = wsum(sy[r] * sq[r]);
    sq[r] -= d * sy[r];
    __syncwarp();
    nq = sqrt(wsum(sq[r] * sq[r]));
  }
  sq[r] /= nq;
  __syncwarp();
  double gy = 0.0, gq = 0.0;   // (G y)_r, (G q)_r
  if (r < m)
    for (int j = 0; j < m; j++) {
      gy = fma(sG[r][j], sy[j], gy);
      gq = fma(sG[r][j], sq[j], gq);
    }
  double g00 = wsum(sy[r] * gy), g01 = wsum(sy[r] * gq), g11 = wsum(sq[r] * gq);
  double g10 = wsum(sq[r] * gy);
  if (r < m) yp[(int64_t)b * M + r] = sq[r];
  if (r == 0) {
    double* Gb = G + (int64_t)b * M * M;
    double off = 0.5 * (g01 + g10);
    Gb[0] = g00;
    Gb[1] = off;
    Gb[M] = off;
    Gb[M + 1] = g11;
  }
}

// In place: V_0 = V y, V_1 = V q, AV_0 = AV y, AV_1 = AV q (q in yp)
__global__ void k_restart_vec(double* __restrict__ V, double* __restrict__ AV, int m, int M,
                              int64_t N, const double* __restrict__ y, const double* __restrict__ q,
                              const int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double sy[32], sq[32];
  if (threadIdx.x < m) {
    sy[threadIdx.x] = y[(int64_t)b * M + threadIdx.x];
    sq[threadIdx.x] = q[(int64_t)b * M + threadIdx.x];
  }
  __syncthreads();
  double* Vb = V + (int64_t)b * M * N;
  double* AVb = AV + (int64_t)b * M * N;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    double x = 0.0, xp = 0.0, ax = 0.0, axp = 0.0;
    for (int i = 0; i < m; i++) {
      double v = Vb[(int64_t)i * N + k], av = AVb[(int64_t)i * N + k];
      x = fma(sy[i], v, x);
      xp = fma(sq[i], v, xp);
      ax = fma(sy[i], av, ax);
      axp = fma(sq[i], av, axp);
    }
    Vb[k] = x;
    Vb[N + k] = xp;
    AVb[k] = ax;
    AVb[N + k] = axp;
  }
}

// y_prev <- y (zero padded), or e_0 right after a restart
__global__ void k_save_yprev(const double* __restrict__ y, int m, int M, int restarted,
                             const int32_t* __restrict__ active, double* __restrict__ yp) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  for (int i = threadIdx.x; i < M; i += blockDim.x)
    yp[(int64_t)b * M + i] = restarted ? (i == 0 ? 1.0 : 0.0) : (i < m ? y[(int64_t)b * M + i] : 0.0);
}

// t = r / (theta - H_II), then (closed shell, nstrb < 0) t <- (t + t^T)/2
// so that every subspace vector stays exactly in the alpha<->beta symmetric
// (even-S) sector; each thread owns the pair (Ia,Ib), (Ib,Ia) with Ia <= Ib.
// A high-spin space (nstrb >= 0 beta strings) has no such symmetry.
__global__ void k_precondition(double* __restrict__ T, const double* __restrict__ hd, int nstr,
                               int nstrb, const double* __restrict__ theta,
                               const int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const double th = theta[b];
  const int64_t N = (int64_t)nstr * (nstrb < 0 ? nstr : nstrb);
  double* Tb = T + (int64_t)b * N;
  const double* hb = hd + (int64_t)b * N;
  if (nstrb >= 0) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
      double d = th - hb[k];
      if (fabs(d) < 1e-8) d = d < 0.0 ? -1e-8 : 1e-8;
      Tb[k] = Tb[k] / d;
    }
    return;
  }
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int ia = (int)(k / nstr), ib = (int)(k % nstr);
    if (ia > ib) continue;
    const int64_t kt = (int64_t)ib * nstr + ia;
    double d1 = th - hb[k], d2 = th - hb[kt];
    if (fabs(d1) < 1e-8) d1 = d1 < 0.0 ? -1e-8 : 1e-8;
    if (fabs(d2) < 1e-8) d2 = d2 < 0.0 ? -1e-8 : 1e-8;
    const double t = 0.5 * (Tb[k] / d1 + Tb[kt] / d2);
    Tb[k] = t;
    Tb[kt] = t;
  }
}

// T -= sum_i coef[i] V[i]
__global__ void k_orth_axpy(double* __restrict__ T, const double* __restrict__ V, int m, int M,
                            int64_t N, const double* __restrict__ coef,
                            const int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  __shared__ double sc[32];
  if (threadIdx.x < m) sc[threadIdx.x] = coef[(int64_t)b * M + threadIdx.x];
  __syncthreads();
  const double* Vb = V + (int64_t)b * M * N;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    double t = T[(int64_t)b * N + k];
    for (int i = 0; i < m; i++) t = fma(-sc[i], Vb[(int64_t)i * N + k], t);
    T[(int64_t)b * N + k] = t;
  }
}

// V[m] = T / ||T||; a tuple whose correction vanished is marked converged
__global__ void k_append(const double* __restrict__ T, double* __restrict__ V, int m, int M,
                         int64_t N, const double* __restrict__ nrm2, int32_t* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  double n2 = nrm2[(int64_t)b * M];
  if (!(n2 > 1e-28)) {
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) active[b] = 2;   // frozen after this pass
    return;
  }
  double inv = 1.0 / sqrt(n2);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    V[(int64_t)b * M * N + (int64_t)m * N + k] = T[(int64_t)b * N + k] * inv;
}

__global__ void k_fix_frozen(int32_t* active, int B) {
  for (int b = threadIdx.x; b < B; b += blockDim.x)
    if (active[b] == 2) active[b] = 0;
}

// start vector: lowest diagonal determinant (Ia, Ib), symmetrised for a
// closed shell (nstrb < 0); for a high-spin space (nstrb beta strings) the
// determinant itself
__global__ void k_guess(const double* __restrict__ hd, int nstr, int nstrb, int M,
                        double* __restrict__ V) {
  const int b = blockIdx.x;
  const int64_t N = (int64_t)nstr * (nstrb < 0 ? nstr : nstrb);
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  double best = 1e300;
  int64_t bi = 0;
  for (int64_t k = threadIdx.x; k < N; k += blockDim.x) {
    double v = hd[(int64_t)b * N + k];
    if (v < best) { best = v; bi = k; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) {
      double o = sv[threadIdx.x + s];
      int64_t oi = si[threadIdx.x + s];
      if (o < sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  double* Vb = V + (int64_t)b * M * N;
  for (int64_t k = threadIdx.x; k < N; k += blockDim.x) Vb[k] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t i0 = si[0];
    int ia = (int)(i0 / nstr), ib = (int)(i0 % nstr);
    if (nstrb >= 0 || ia == ib) Vb[i0] = 1.0;
    else {
      Vb[(int64_t)ia * nstr + ib] = sqrt(0.5);
      Vb[(int64_t)ib * nstr + ia] = sqrt(0.5);
    }
  }
}

__global__ void k_fill(double* __restrict__ v, int n, double x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = x;
}

__global__ void k_set_i32(int32_t* __restrict__ v, int n, int32_t x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = x;
}

}  // namespace

struct Multidot {
  DevBuf<double> partial;
  int nchunks = 0;
  // out[b*out_bstride + i*out_istride] = X[b][i] . Y[b], i < m
  void run(mbe_ctx* ctx, const double* X, int64_t xb, int64_t xv, const double* Y, int64_t yb,
           int m, int64_t N, int B, const int32_t* active, double* out, int64_t ob, int64_t oi) {
    nchunks = (int)((N + DOT_CHUNK - 1) / DOT_CHUNK);
    size_t need = (size_t)B * m * nchunks;
    if (partial.n < need) partial.reset(&ctx->pool, need);
    dim3 g(nchunks, B);
    k_multidot_partial<<<g, 256, 0, ctx->stream>>>(X, xb, xv, Y, yb, m, N, nchunks, active,
                                                   partial.ptr);
    CU_LAUNCH_CHECK();
    k_multidot_final<<<B, 32, 0, ctx->stream>>>(partial.ptr, m, nchunks, active, out, ob, oi);
    CU_LAUNCH_CHECK();
  }
};

// Davidson for one batch of tuples: one stage with FP64 (or emulated-FP64)
// sigma vectors to conv_tol_r / conv_tol_e.
void davidson_batch(mbe_ctx* ctx, BinProblem& bp, double* e_out_host, int32_t* status_host,
                    double* s2_host, double* x_out_dev, const GuessPlan* plan) {
  const int B = bp.B;
  const int M = std::max(4, std::min(32, ctx->opt.max_subspace));
  const int64_t N = bp.ndet;
  const double shift = ctx->opt.spin_shift;
  DevPool* P = &ctx->pool;
  DevBuf<double> V(P, (size_t)B * M * N), AV(P, (size_t)B * M * N), hd(P, (size_t)B * N),
      T(P, (size_t)B * N), Xown(P, x_out_dev ? 0 : (size_t)B * N), G(P, (size_t)B * M * M),
      y(P, (size_t)B * M), yp(P, (size_t)B * M), theta(P, B), theta_old(P, B), rnorm(P, B),
      tolr(P, B), coef(P, (size_t)B * M), xx(P, (size_t)B * M),
      rpart(P, (size_t)B * ((N + DOT_CHUNK - 1) / DOT_CHUNK));
  DevBuf<int32_t> active(P, B), iters(P, B), nact(P, 1);
  double* X = x_out_dev ? x_out_dev : Xown.ptr;
  SigmaWork sw;
  Multidot md;
  cudaStream_t st = ctx->stream;
  // sigma vectors: FP64 CUDA cores (MBE_FP64) or the FP64-grade sliced
  // tensor-core contraction (MBE_EMULATED_FP64, and the mixed mode's
  // fallback for spaces the fused tensor-core kernel does not cover)
  const bool emulated = ctx->opt.precision != MBE_FP64 && ozaki_supported(bp.npair);

  launch_hdiag(ctx, bp, shift, hd.ptr);
  const int nstrb_arg = bp.closed() ? -1 : bp.nstrb;
  k_guess<<<B, 256, 0, st>>>(hd.ptr, bp.nstr, nstrb_arg, M, V.ptr);
  CU_LAUNCH_CHECK();
  if (plan) launch_parent_guess(ctx, *plan, bp.n, bp.nsig, bp.nstr, nullptr, V.ptr, (int64_t)M * N);
  k_set_i32<<<1, 256, 0, st>>>(active.ptr, B, 1);
  CU_LAUNCH_CHECK();
  CU_CHECK(cudaMemsetAsync(iters.ptr, 0, sizeof(int32_t) * B, st));
  CU_CHECK(cudaMemsetAsync(G.ptr, 0, sizeof(double) * B * M * M, st));
  k_fill<<<1, 256, 0, st>>>(tolr.ptr, B, ctx->opt.conv_tol_r);
  CU_LAUNCH_CHECK();

  int64_t eblocks = std::min<int64_t>((N + 255) / 256, 1024);
  dim3 ge((unsigned)eblocks, B);
  const int nchunks = (int)((N + DOT_CHUNK - 1) / DOT_CHUNK);
  dim3 gc(nchunks, B);
  const int max_iter = std::max(1, ctx->opt.max_iter);
  int64_t vecs_tc = 0, vecs_64 = 0;
  int total_it = 0;

  auto sigma = [&](bool /*unused*/, const double* c, double* out) {
    sigma_fp64(ctx, bp, sw, c, (int64_t)M * N, out, (int64_t)M * N, active.ptr, shift, emulated,
               true);
  };
  // precondition the residual in T, orthogonalise it against V[0..m) and
  // append it as V[m] (tuples whose correction vanished are frozen)
  auto extend = [&](int m) {
    k_precondition<<<ge, 256, 0, st>>>(T.ptr, hd.ptr, bp.nstr, nstrb_arg, theta.ptr, active.ptr);
    CU_LAUNCH_CHECK();
    for (int pass = 0; pass < 2; pass++) {
      md.run(ctx, V.ptr, (int64_t)M * N, N, T.ptr, N, m, N, B, active.ptr, coef.ptr, M, 1);
      k_orth_axpy<<<ge, 256, 0, st>>>(T.ptr, V.ptr, m, M, N, coef.ptr, active.ptr);
      CU_LAUNCH_CHECK();
    }
    md.run(ctx, T.ptr, N, 0, T.ptr, N, 1, N, B, active.ptr, coef.ptr, M, 1);
    k_append<<<ge, 256, 0, st>>>(T.ptr, V.ptr, m, M, N, coef.ptr, active.ptr);
    CU_LAUNCH_CHECK();
    k_fix_frozen<<<1, 256, 0, st>>>(active.ptr, B);
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
      fprintf(stderr, "[mbe davidson] n=%d nsig=%d B=%d it=%d active=%d max|r|=%.3e theta0=%.12f\n",
              bp.n, bp.nsig, B, total_it, n, mx, th[0]);
    }
    return n;
  };

  // One stage of Davidson iterations from the current (V, AV, G): the
  // subspace holds m_start vectors and the newest one's sigma is pending.
  // exact0: V_0 carries an exact (FP64) A V_0; its couplings G_0j are then
  // taken as (A V_0).V_j, which involves no reduced-precision sigma, and the
  // stage ends before a restart would replace V_0.
  auto stage = [&](bool use_tc, double tol_e, int rel, int m_start, int cap, int nact0,
                   bool exact0) {
    int m = m_start;
    int nact_h = nact0;
    for (int it = 0; it < cap && total_it < max_iter; it++, total_it++) {
      sigma(use_tc, V.ptr + (int64_t)(m - 1) * N, AV.ptr + (int64_t)(m - 1) * N);
      (use_tc ? vecs_tc : vecs_64) += nact_h;
      md.run(ctx, V.ptr, (int64_t)M * N, N, AV.ptr + (int64_t)(m - 1) * N, (int64_t)M * N, m, N,
             B, active.ptr, coef.ptr, M, 1);
      if (exact0) {
        md.run(ctx, AV.ptr, (int64_t)M * N, 0, V.ptr + (int64_t)(m - 1) * N, (int64_t)M * N, 1, N,
               B, active.ptr, coef.ptr, M, 1);
      }
      k_store_grow<<<B, 32, 0, st>>>(coef.ptr, m, M, active.ptr, G.ptr);
      CU_LAUNCH_CHECK();
      k_jacobi<<<B, 32, 0, st>>>(G.ptr, m, M, active.ptr, theta.ptr, y.ptr);
      CU_LAUNCH_CHECK();
      k_residual<<<gc, 256, 0, st>>>(V.ptr, AV.ptr, m, M, N, y.ptr, theta.ptr, active.ptr, X,
                                     T.ptr, nchunks, rpart.ptr);
      CU_LAUNCH_CHECK();
      k_converge<<<1, 256, 0, st>>>(rpart.ptr, nchunks, B, m_start > 1 ? it + 1 : it, tolr.ptr,
                                    tol_e, rel, theta.ptr, theta_old.ptr, rnorm.ptr, active.ptr,
                                    iters.ptr, nact.ptr);
      CU_LAUNCH_CHECK();
      nact_h = count_active();
      if (nact_h == 0) return;
      if (exact0 && m == M) return;   // the next exact point restarts
      int restarted = 0;
      if (m == M) {   // restart with {x, x_prev}
        k_restart_coef<<<B, 32, 0, st>>>(y.ptr, yp.ptr, m, M, active.ptr, G.ptr);
        CU_LAUNCH_CHECK();
        k_restart_vec<<<ge, 256, 0, st>>>(V.ptr, AV.ptr, m, M, N, y.ptr, yp.ptr, active.ptr);
        CU_LAUNCH_CHECK();
        m = 2;
        restarted = 1;
      }
      k_save_yprev<<<B, 32, 0, st>>>(y.ptr, m, M, restarted, active.ptr, yp.ptr);
      CU_LAUNCH_CHECK();
      extend(m);
      m++;
    }
  };

  stage(false, ctx->opt.conv_tol_e, 0, 1, max_iter, B, false);
  if (emulated && sigma_tc_error(ctx, sw))
    throw MbeError{MBE_ETIMEOUT, "tensor-core contraction wait timed out"};

  // status and energies: eps = E_core + theta - shift <x|S^2|x> / <x|x>
  std::vector<int32_t> it_h(B);
  std::vector<double> rn_h(B);
  CU_CHECK(cudaMemcpyAsync(it_h.data(), iters.ptr, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(rn_h.data(), rnorm.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  s2_apply(ctx, bp, X, N, T.ptr, N, nullptr);
  md.run(ctx, X, N, 0, T.ptr, N, 1, N, B, nullptr, coef.ptr, 1, 1);
  md.run(ctx, X, N, 0, X, N, 1, N, B, nullptr, xx.ptr, 1, 1);
  std::vector<double> th(B), s2(B), ec(B), nx(B);
  CU_CHECK(cudaMemcpyAsync(th.data(), theta.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(s2.data(), coef.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(nx.data(), xx.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaMemcpyAsync(ec.data(), bp.ecore.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  CU_CHECK(cudaStreamSynchronize(st));
  const double rtol = ctx->opt.conv_tol_r;
  for (int b = 0; b < B; b++) {
    const double s2n = nx[b] > 0.0 ? s2[b] / nx[b] : 0.0;
    if (e_out_host) e_out_host[b] = ec[b] + th[b] - shift * s2n;
    if (s2_host) s2_host[b] = s2n;
    bool ok = rn_h[b] <= rtol * 10.0 || N == 1;
    if (status_host) status_host[b] = ok ? MBE_OK : MBE_ENOCONV;
    ctx->stats.iters_total += it_h[b];
    ctx->stats.iters_max = std::max<int64_t>(ctx->stats.iters_max, it_h[b]);
    ctx->stats.noconv += ok ? 0 : 1;
  }
  const double per = 2.0 * (double)N * bp.npair * bp.npair;
  ctx->stats.casci += B;
  ctx->stats.sigma_vectors += vecs_tc + vecs_64;
  ctx->stats.sigma_flops += (double)(vecs_tc + vecs_64) * per;
  ctx->stats.fp64_flops += (double)(vecs_tc + vecs_64) * per;   // exact sigma vectors
}
