// Lowest eigenpair of the Davidson subspace matrix (the Rayleigh-Ritz step),
// one warp per tuple.
//
// GB300 issues FP64 at a small fraction of its FP32 rate, so the O(m^3)
// diagonalisation runs in FP32 and only O(m^2) work per step is FP64:
//   1. cyclic Jacobi in FP32 with the round-robin (tournament) ordering: the
//      m/2 rotations of one step touch disjoint index pairs and are applied
//      together (columns, then rows), so every lane works on every step;
//   2. the lowest FP32 eigenvector z_k is refined in FP64 by Newton steps in
//      the approximate eigenbasis: with s = G y - theta y (FP64),
//        y <- y - sum_{j != k} z_j (z_j . s) / (lambda_j - theta),
//      each step multiplying the error by ~ (FP32 residual of Z) / gap, and
//      theta = y.G.y is the FP64 Rayleigh quotient of the normalised y.
// m <= 32; G is read symmetrised, (G + G^T) / 2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct RitzShared {
  float A[32][33];
  float Z[32][33];
  double G[32][33];
  float cs[16][2];
  int pq[16][2];
  float lam[32];
  float s32[32];
  float coef[32];
};

__device__ __forceinline__ double ritz_warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float ritz_warp_sumf(float v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Called by all 32 lanes of one warp.  Gb: row-major, leading dimension M.
static __device__ void ritz_lowest(const double* __restrict__ Gb, int m, int M, RitzShared& S,
                            double* theta_out, double* y_out) {
  const int r = threadIdx.x & 31;
  for (int i = 0; i < m; i++)
    if (r < m) {
      const double g = 0.5 * (Gb[(int64_t)i * M + r] + Gb[(int64_t)r * M + i]);
      S.G[i][r] = g;
      S.A[i][r] = (float)g;
      S.Z[i][r] = (i == r) ? 1.f : 0.f;
    }
  __syncwarp();
  // ---- 1. FP32 tournament Jacobi
  const int n2 = m + (m & 1);
  for (int sweep = 0; sweep < 12 && m > 1; sweep++) {
    float off = 0.f, dia = 0.f;
    if (r < m)
      for (int j = 0; j < m; j++) {
        const float a = S.A[r][j];
        if (j != r) off += a * a;
        else dia += a * a;
      }
    off = ritz_warp_sumf(off);
    dia = ritz_warp_sumf(dia);
    if (off <= 1e-12f * dia) break;
    for (int step = 0; step < n2 - 1; step++) {
      if (r < n2 / 2) {
        auto pos = [&](int j) { return j == 0 ? 0 : 1 + (j - 1 + step) % (n2 - 1); };
        int p = pos(r), q = pos(n2 - 1 - r);
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < m) {
          const float apq = S.A[p][q];
          if (fabsf(apq) > 1e-30f) {
            const float th = (S.A[q][q] - S.A[p][p]) / (2.f * apq);
            const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
            c = rsqrtf(t * t + 1.f);
            s = t * c;
          }
        }
        S.pq[r][0] = p;
        S.pq[r][1] = q < m ? q : -1;
        S.cs[r][0] = c;
        S.cs[r][1] = s;
      }
      __syncwarp();
      // columns: A <- A J, Z <- Z J (lane = row)
      if (r < m)
        for (int i = 0; i < n2 / 2; i++) {
          const int p = S.pq[i][0], q = S.pq[i][1];
          if (q < 0) continue;
          const float c = S.cs[i][0], s = S.cs[i][1];
          const float a = S.A[r][p], b = S.A[r][q];
          S.A[r][p] = c * a - s * b;
          S.A[r][q] = s * a + c * b;
          const float za = S.Z[r][p], zb = S.Z[r][q];
          S.Z[r][p] = c * za - s * zb;
          S.Z[r][q] = s * za + c * zb;
        }
      __syncwarp();
      // rows: A <- J^T A (lane = column)
      if (r < m)
        for (int i = 0; i < n2 / 2; i++) {
          const int p = S.pq[i][0], q = S.pq[i][1];
          if (q < 0) continue;
          const float c = S.cs[i][0], s = S.cs[i][1];
          const float a = S.A[p][r], b = S.A[q][r];
          S.A[p][r] = c * a - s * b;
          S.A[q][r] = s * a + c * b;
        }
      __syncwarp();
    }
  }
  if (r < m) S.lam[r] = S.A[r][r];
  __syncwarp();
  int k = 0;
  for (int i = 1; i < m; i++)
    if (S.lam[i] < S.lam[k]) k = i;
  // ---- 2. FP64 Newton refinement of the lowest pair
  double y = r < m ? (double)S.Z[r][k] : 0.0;
  double nn = ritz_warp_sum(y * y);
  y /= sqrt(nn);
  double theta = 0.0;
  for (int it = 0; it < 4; it++) {
    double gy = 0.0;
    for (int j = 0; j < m; j++) {
      const double yj = __shfl_sync(0xffffffffu, y, j);
      if (r < m) gy = fma(S.G[r][j], yj, gy);
    }
    theta = ritz_warp_sum(y * gy);
    if (it == 3) break;
    S.s32[r] = (float)(gy - theta * y);
    __syncwarp();
    float cf = 0.f;
    if (r < m && r != k) {
      const float den = S.lam[r] - (float)theta;
      if (fabsf(den) > 1e-6f * fmaxf(1.f, fabsf((float)theta))) {
        float d = 0.f;
        for (int j = 0; j < m; j++) d = fmaf(S.Z[j][r], S.s32[j], d);
        cf = d / den;
      }
    }
    S.coef[r] = cf;
    __syncwarp();
    float w = 0.f;
    if (r < m)
      for (int j = 0; j < m; j++) w = fmaf(S.Z[r][j], S.coef[j], w);
    y -= (double)w;
    nn = ritz_warp_sum(y * y);
    y /= sqrt(nn);
    __syncwarp();
  }
  if (r == 0) *theta_out = theta;
  if (r < m) y_out[r] = y;
}
