// P-space preconditioner of the mixed-precision Davidson iteration.
//
// The diagonal (Davidson) preconditioner t_I = r_I / (theta - A_II) treats
// every determinant alone.  The determinants of lowest diagonal energy are
// the ones that couple most strongly to the solution and among themselves,
// so for a set P of them the correction is taken with the exact block:
//   t_P = (theta - A_PP)^{-1} r_P,     t_I = r_I / (theta - A_II) elsewhere,
// A = H + lambda S^2 (the operator of the Davidson iteration, core energy
// excluded).  Every Davidson vector is alpha-beta symmetric, so P is a set
// of symmetric basis functions: a canonical determinant pair (a, b), a <= b,
// stands for (|a b> + |b a>) / sqrt(2) (or |a a>), and A_PP is A in that
// basis.  Per tuple, once:
//   k_psp_select  the npp canonical pairs of lowest diagonal (radix select on
//                 the FP32 diagonal, ties broken by index), in index order;
//   k_psp_eigh    A_PP from the Slater-Condon rules (one-electron h_eff with
//                 the core folded in, (pq|rs) of the active orbitals, the
//                 spin-exchange couplings of lambda S^2), then its
//                 eigenvectors by cyclic Jacobi (parallel tournament order)
//                 in shared memory, FP32 (a preconditioner needs no more);
// per iteration:
//   k_psp_apply   t_P = U (theta - Lambda)^{-1} U^T r_P (r_P recovered from
//                 the diagonal correction as t_I (theta - A_II)), written
//                 back into the packed vector, and the first Gram-Schmidt pass's
//                 dot products corrected for the changed elements; the same
//                 for M^-1 x, x the Ritz vector.
// With an exact block M^-1 r = -x on P whenever x lies in P and does not
// couple out of it (the lowest-diagonal start vector of a small space does),
// which the orthogonalisation removes, so the Davidson iteration takes
// Olsen's combination t = M^-1 r - eps M^-1 x, eps = x.M^-1 r / x.M^-1 x
// (J. Olsen, P. Jorgensen, J. Simons, Chem. Phys. Lett. 169, 463 (1990)),
// an inverse-iteration step in that case.  npp is capped at half the
// canonical pairs.
#include "mbe_internal.cuh"
#include <algorithm>

namespace {

constexpr int PSP_MAX = 128;
constexpr int PSP_PITCH = PSP_MAX + 1;   // row pitch of the shared matrices
constexpr int SEL_THREADS = 1024;
constexpr int EIG_THREADS = 1024;
constexpr int APPLY_THREADS = 256;
constexpr int EIG_SWEEPS = 10;

// FP32 bit pattern mapped to an unsigned key with the same order
__device__ __forceinline__ uint32_t order_key(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// exclusive count of set flags below this thread in the block, and the
// block total (all threads must call; s_warp holds 32 ints)
__device__ __forceinline__ int block_flag_scan(bool f, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_warp[warp] = __popc(bal);
  __syncthreads();
  int off = 0, tot = 0;
  const int nw = (int)(blockDim.x >> 5);
  for (int w = 0; w < nw; w++) {
    const int c = s_warp[w];
    if (w < warp) off += c;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return off + __popc(bal & ((1u << lane) - 1u));
}

// psel[b][0..npp) = linear indices a nstr + c (a <= c) of the npp canonical
// pairs of lowest diagonal, in increasing index order (the diagonal and all
// vectors are in the packed symmetric layout, element (a, c) at
// sym_index(a, c))
__global__ void __launch_bounds__(SEL_THREADS)
    k_psp_select(const float* __restrict__ hd_all, int nstr, int64_t ld, int npp,
                 int32_t* __restrict__ psel) {
  const int b = blockIdx.x;
  const int64_t N = (int64_t)nstr * nstr;
  const float* hd = hd_all + (int64_t)b * ld;
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix;
  __shared__ int s_k;
  __shared__ int s_warp[32];
  uint32_t prefix = 0, mask = 0;
  int k = npp;   // rank (from 1) of the threshold key among the remaining keys
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
      const int a = (int)(i / nstr), c = (int)(i - (int64_t)a * nstr);
      if (a > c) continue;
      const uint32_t key = order_key(hd[sym_index(a, c, nstr)]);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t cum = 0;
      int d = 0;
      for (; d < 255; d++) {
        if (cum + hist[d] >= (uint32_t)k) break;
        cum += hist[d];
      }
      s_k = k - (int)cum;
      s_prefix = prefix | ((uint32_t)d << shift);
    }
    __syncthreads();
    prefix = s_prefix;
    k = s_k;
    mask |= 0xFFu << shift;
    __syncthreads();
  }
  // keys below the threshold, then the first k equal to it, in index order
  const uint32_t thr = prefix;
  const int need_eq = k;
  int base = 0, base_eq = 0;
  for (int64_t i0 = 0; i0 < N && base < npp; i0 += blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    bool lt = false, eq = false;
    if (i < N) {
      const int a = (int)(i / nstr), c = (int)(i - (int64_t)a * nstr);
      if (a <= c) {
        const uint32_t key = order_key(hd[sym_index(a, c, nstr)]);
        lt = key < thr;
        eq = key == thr;
      }
    }
    int teq = 0, tsel = 0;
    const int req = base_eq + block_flag_scan(eq, s_warp, &teq);
    const bool sel = lt || (eq && req < need_eq);
    const int pos = base + block_flag_scan(sel, s_warp, &tsel);
    if (sel && pos < npp) psel[(int64_t)b * PSP_MAX + pos] = (int)i;
    base += tsel;
    base_eq += teq;
  }
}

__device__ __forceinline__ int pair_index(int p, int q) {
  return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p;
}

// phase of a+_p a_q on the string m (q occupied, p empty): the parity of the
// occupied orbitals strictly between p and q
__device__ __forceinline__ float exc_sign(uint32_t m, int p, int q) {
  const int lo = min(p, q), hi = max(p, q);
  const uint32_t between = m & ((1u << hi) - 1u) & ~((2u << lo) - 1u);
  return (__popc(between) & 1) ? -1.f : 1.f;
}

// <na nb| H + lam S^2 |ma mb> for two different determinants (Slater-Condon
// rules; g holds (pq|rs) packed by orbital pairs, heff the one-electron
// operator with the core folded in)
__device__ float psp_offdiag(uint32_t ma, uint32_t mb, uint32_t na, uint32_t nb,
                             const float* heff, const float* g, int n, int npair, float lam) {
  const uint32_t da = ma ^ na, db = mb ^ nb;
  const int ea = __popc(da) >> 1, eb = __popc(db) >> 1;
  if (ea + eb > 2 || ea + eb == 0) return 0.f;
  auto G = [&](int p, int q, int r, int s) { return g[pair_index(p, q) * npair + pair_index(r, s)]; };
  if (ea + eb == 1) {
    // single excitation q -> p in one spin; the other spin's occupied
    // orbitals enter through the Coulomb term only
    const uint32_t m = ea ? ma : mb, nm = ea ? na : nb, d = ea ? da : db;
    const uint32_t other = ea ? mb : ma;
    const int q = __ffs(m & d) - 1, p = __ffs(nm & d) - 1;
    float v = heff[p * n + q];
    for (uint32_t k = m; k; k &= k - 1) {
      const int o = __ffs(k) - 1;
      v += G(p, q, o, o) - G(p, o, o, q);
    }
    for (uint32_t k = other; k; k &= k - 1) {
      const int o = __ffs(k) - 1;
      v += G(p, q, o, o);
    }
    return exc_sign(m, p, q) * v;
  }
  if (ea == 1 && eb == 1) {
    const int q = __ffs(ma & da) - 1, p = __ffs(na & da) - 1;
    const int s = __ffs(mb & db) - 1, r = __ffs(nb & db) - 1;
    const float sg = exc_sign(ma, p, q) * exc_sign(mb, r, s);
    float v = sg * G(p, q, r, s);
    if (p == s && q == r) v -= lam * sg;   // spin exchange (S^2 coupling)
    return v;
  }
  // same-spin double: holes q < s, particles p < r
  const uint32_t m = ea ? ma : mb, nm = ea ? na : nb, d = ea ? da : db;
  const uint32_t hm = m & d, pm = nm & d;
  const int q = __ffs(hm) - 1, s = 31 - __clz(hm);
  const int p = __ffs(pm) - 1, r = 31 - __clz(pm);
  const float s1 = exc_sign(m, p, q);
  const uint32_t m1 = m ^ (1u << p) ^ (1u << q);
  const float s2 = exc_sign(m1, r, s);
  return s1 * s2 * (G(p, q, r, s) - G(p, s, r, q));
}

struct EigShared {
  uint32_t a_off, u_off, g_off, h_off, total;
};

__host__ __device__ inline EigShared eig_layout(int n) {
  const int npair = n * (n + 1) / 2;
  EigShared s;
  uint32_t o = 0;
  s.a_off = o;
  o += PSP_MAX * PSP_PITCH * 4;
  s.u_off = o;
  o += PSP_MAX * PSP_PITCH * 4;
  s.g_off = o;
  o += (uint32_t)npair * npair * 4;
  s.h_off = o;
  o += (uint32_t)n * n * 4;
  s.total = o;
  return s;
}

// A_PP in the symmetric basis and its eigenpairs: lam_out[b][k], U[b][u][k]
// (column k the eigenvector of lam_k)
__global__ void __launch_bounds__(EIG_THREADS)
    k_psp_eigh(const uint32_t* __restrict__ masks, int nstr, int n, int nsig,
               const double* __restrict__ heff_all, const double* __restrict__ hp_all,
               const double* __restrict__ gp_all, const float* __restrict__ hd_all, int64_t ld,
               float lam, int npp, const int32_t* __restrict__ psel, float* __restrict__ lam_out,
               float* __restrict__ U_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x;
  const int npair = n * (n + 1) / 2;
  const EigShared L = eig_layout(n);
  float* A = (float*)(smem + L.a_off);
  float* U = (float*)(smem + L.u_off);
  float* g = (float*)(smem + L.g_off);
  float* heff = (float*)(smem + L.h_off);
  __shared__ uint32_t s_ma[PSP_MAX], s_mb[PSP_MAX];
  __shared__ int s_diag[PSP_MAX];
  __shared__ float s_hd[PSP_MAX];
  __shared__ float s_c[PSP_MAX / 2], s_s[PSP_MAX / 2];
  __shared__ int s_p[PSP_MAX / 2], s_q[PSP_MAX / 2];
  __shared__ float s_red[32];
  __shared__ int s_done;
  const int tid = threadIdx.x;
  // (pq|rs) = g'_PQ - (h'_pq d_rs + d_pq h'_rs) / N_active (the definition of g')
  const double* gp = gp_all + (int64_t)b * npair * npair;
  const double* hp = hp_all + (int64_t)b * n * n;
  const double inv = nsig > 0 ? 1.0 / (2 * nsig) : 0.0;
  for (int t = tid; t < npair * npair; t += blockDim.x) {
    const int P = t / npair, Q = t - P * npair;
    int p = 0;
    while ((p + 1) * (p + 2) / 2 <= P) p++;
    const int q = P - p * (p + 1) / 2;
    int r = 0;
    while ((r + 1) * (r + 2) / 2 <= Q) r++;
    const int s = Q - r * (r + 1) / 2;
    double v = gp[t];
    if (r == s) v -= hp[p * n + q] * inv;
    if (p == q) v -= hp[r * n + s] * inv;
    g[t] = (float)v;
  }
  for (int t = tid; t < n * n; t += blockDim.x) heff[t] = (float)heff_all[(int64_t)b * n * n + t];
  // basis functions: canonical pairs (a, c), a <= c
  for (int u = tid; u < npp; u += blockDim.x) {
    const int i = psel[(int64_t)b * PSP_MAX + u];
    const int a = i / nstr, c = i - a * nstr;
    s_ma[u] = masks[a];
    s_mb[u] = masks[c];
    s_diag[u] = a == c;
    s_hd[u] = hd_all[(int64_t)b * ld + sym_index(a, c, nstr)];
  }
  // an odd npp gets one decoupled pad index (zero row and column)
  const int m = (npp + 1) & ~1;
  for (int t = tid; t < PSP_MAX * PSP_PITCH; t += blockDim.x) {
    A[t] = 0.f;
    U[t] = 0.f;
  }
  __syncthreads();
  const float r2 = 0.70710678118654752f;
  for (int t = tid; t < npp * npp; t += blockDim.x) {
    const int u = t / npp, v = t - u * npp;
    if (v < u) continue;
    // |u> = c_u (|a b> + |b a>) (one term when a == b), c_u = 1/sqrt(2) or 1
    const uint32_t ua = s_ma[u], ub = s_mb[u], va = s_ma[v], vb = s_mb[v];
    float x;
    if (u == v) {
      x = s_diag[u] ? s_hd[u] : s_hd[u] + psp_offdiag(ua, ub, ub, ua, heff, g, n, npair, lam);
    } else {
      float sum = psp_offdiag(ua, ub, va, vb, heff, g, n, npair, lam);
      if (!s_diag[v]) sum += psp_offdiag(ua, ub, vb, va, heff, g, n, npair, lam);
      if (!s_diag[u]) {
        sum += psp_offdiag(ub, ua, va, vb, heff, g, n, npair, lam);
        if (!s_diag[v]) sum += psp_offdiag(ub, ua, vb, va, heff, g, n, npair, lam);
      }
      x = sum * (s_diag[u] ? 1.f : r2) * (s_diag[v] ? 1.f : r2);
    }
    A[u * PSP_PITCH + v] = x;
    A[v * PSP_PITCH + u] = x;
  }
  for (int u = tid; u < m; u += blockDim.x) U[u * PSP_PITCH + u] = 1.f;
  __syncthreads();
  // cyclic Jacobi, tournament order: in round r the m/2 disjoint pairs
  // (pos(j), pos(m-1-j)) with position 0 fixed and the others rotating
  for (int sweep = 0; sweep < EIG_SWEEPS; sweep++) {
    for (int round = 0; round < m - 1; round++) {
      if (tid < m / 2) {
        auto pos = [&](int k) { return k == 0 ? 0 : 1 + (k - 1 + round) % (m - 1); };
        int p = pos(tid), q = pos(m - 1 - tid);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const float app = A[p * PSP_PITCH + p], aqq = A[q * PSP_PITCH + q];
        const float apq = A[p * PSP_PITCH + q];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) > 1e-30f) {
          const float tau = (aqq - app) / (2.f * apq);
          const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = rsqrtf(1.f + t * t);
          s = t * c;
        }
        s_p[tid] = p;
        s_q[tid] = q;
        s_c[tid] = c;
        s_s[tid] = s;
      }
      __syncthreads();
      // rows p, q of A <- J^T A
      for (int t = tid; t < (m / 2) * m; t += blockDim.x) {
        const int j = t / m, col = t - j * m;
        const int p = s_p[j], q = s_q[j];
        const float c = s_c[j], s = s_s[j];
        const float x = A[p * PSP_PITCH + col], y = A[q * PSP_PITCH + col];
        A[p * PSP_PITCH + col] = c * x - s * y;
        A[q * PSP_PITCH + col] = s * x + c * y;
      }
      __syncthreads();
      // columns p, q of A and U <- A J, U J
      for (int t = tid; t < (m / 2) * m; t += blockDim.x) {
        const int j = t / m, row = t - j * m;
        const int p = s_p[j], q = s_q[j];
        const float c = s_c[j], s = s_s[j];
        const float x = A[row * PSP_PITCH + p], y = A[row * PSP_PITCH + q];
        A[row * PSP_PITCH + p] = c * x - s * y;
        A[row * PSP_PITCH + q] = s * x + c * y;
        const float ux = U[row * PSP_PITCH + p], uy = U[row * PSP_PITCH + q];
        U[row * PSP_PITCH + p] = c * ux - s * uy;
        U[row * PSP_PITCH + q] = s * ux + c * uy;
      }
      __syncthreads();
    }
    // off-diagonal against diagonal weight
    float off = 0.f, dia = 0.f;
    for (int t = tid; t < m * m; t += blockDim.x) {
      const int i = t / m, j = t - i * m;
      const float x = A[i * PSP_PITCH + j];
      if (i == j) dia += x * x;
      else off += x * x;
    }
    for (int o = 16; o; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      dia += __shfl_down_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) s_red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      float so = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) so += s_red[w];
      s_red[0] = so;
    }
    __syncthreads();
    const float so = s_red[0];
    __syncthreads();
    if ((tid & 31) == 0) s_red[tid >> 5] = dia;
    __syncthreads();
    if (tid == 0) {
      float sd = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) sd += s_red[w];
      s_done = so <= 1e-10f * sd;   // off-diagonal ~1e-5 of the diagonal
    }
    __syncthreads();
    if (s_done) break;
  }
  for (int k = tid; k < npp; k += blockDim.x) lam_out[(int64_t)b * PSP_MAX + k] = A[k * PSP_PITCH + k];
  float* Ub = U_out + (int64_t)b * PSP_MAX * PSP_MAX;
  for (int t = tid; t < npp * npp; t += blockDim.x) {
    const int u = t / npp, k = t - u * npp;
    Ub[u * PSP_MAX + k] = U[u * PSP_PITCH + k];
  }
}

// t_P = U (theta - Lambda)^{-1} U^T r_P for the tuples still iterating; with
// fix_dots the first Gram-Schmidt pass's partial dot products (chunk 0 of
// `partial`) take the change of t.  With olsen the same block solve turns
// u = x / (theta - A_II) (Uo, from the residual kernel) into M^-1 x on P,
// and the partial sums x.t, x.u (xpart) and, with fix_dots, V.u (upart)
// take their changes.
__global__ void __launch_bounds__(APPLY_THREADS)
    k_psp_apply(float* __restrict__ T, const float* __restrict__ hd_all, int nstr, int64_t ld,
                const double* __restrict__ theta, int npp, const int32_t* __restrict__ psel,
                const float* __restrict__ U_all, const float* __restrict__ lam_all,
                const float* __restrict__ V, int m, int M, int nchunks,
                double* __restrict__ partial, int fix_dots, const int32_t* __restrict__ active,
                int olsen, float* __restrict__ Uo, const float* __restrict__ X,
                double* __restrict__ upart, double* __restrict__ xpart) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  extern __shared__ __align__(16) unsigned char smem[];
  float* sU = (float*)smem;   // npp x npp, pitch PSP_PITCH
  __shared__ float s_r[PSP_MAX], s_x[PSP_MAX], s_w[PSP_MAX], s_wx[PSP_MAX];
  __shared__ float s_del[PSP_MAX], s_delu[PSP_MAX], s_xv[PSP_MAX];
  __shared__ int s_i[PSP_MAX];
  const int tid = threadIdx.x;
  float* Tb = T + (int64_t)b * ld;
  float* Ob = olsen ? Uo + (int64_t)b * ld : nullptr;
  const float* Xb = olsen ? X + (int64_t)b * ld : nullptr;
  const float* hb = hd_all + (int64_t)b * ld;
  const float th = (float)theta[b];
  const float* Ub = U_all + (int64_t)b * PSP_MAX * PSP_MAX;
  for (int t = tid; t < npp * npp; t += blockDim.x) {
    const int u = t / npp, k = t - u * npp;
    sU[u * PSP_PITCH + k] = Ub[u * PSP_MAX + k];
  }
  const float sq2 = 1.41421356237309505f, r2 = 0.70710678118654752f;
  for (int u = tid; u < npp; u += blockDim.x) {
    const int i0 = psel[(int64_t)b * PSP_MAX + u];
    const int a = i0 / nstr, c = i0 - a * nstr;
    const int i = (int)sym_index(a, c, nstr);          // packed position
    // the diagonal correction's denominator, exactly as the residual kernel
    float d = th - hb[i];
    if (fabsf(d) < 1e-4f) d = d < 0.f ? -1e-4f : 1e-4f;
    const float r = Tb[i] * d;
    s_r[u] = a == c ? r : sq2 * r;
    if (olsen) {
      const float x = Xb[i];
      s_xv[u] = x;
      s_x[u] = a == c ? x : sq2 * x;
    }
    s_i[u] = i;
  }
  __syncthreads();
  for (int k = tid; k < npp; k += blockDim.x) {
    float w = 0.f, wx = 0.f;
    for (int u = 0; u < npp; u++) {
      const float uk = sU[u * PSP_PITCH + k];
      w = fmaf(uk, s_r[u], w);
      if (olsen) wx = fmaf(uk, s_x[u], wx);
    }
    float dl = th - lam_all[(int64_t)b * PSP_MAX + k];
    if (fabsf(dl) < 1e-4f) dl = dl < 0.f ? -1e-4f : 1e-4f;
    s_w[k] = w / dl;
    s_wx[k] = wx / dl;
  }
  __syncthreads();
  for (int u = tid; u < npp; u += blockDim.x) {
    float y = 0.f, yx = 0.f;
    for (int k = 0; k < npp; k++) {
      const float uk = sU[u * PSP_PITCH + k];
      y = fmaf(uk, s_w[k], y);
      if (olsen) yx = fmaf(uk, s_wx[k], yx);
    }
    const int i = s_i[u];
    const bool diag = i < sym_nd(nstr);
    const float f = diag ? 1.f : 2.f;   // both elements of a pair change alike
    const float tn = diag ? y : y * r2;
    s_del[u] = (tn - Tb[i]) * f;
    Tb[i] = tn;
    if (olsen) {
      const float un = diag ? yx : yx * r2;
      s_delu[u] = (un - Ob[i]) * f;
      Ob[i] = un;
    }
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  if (olsen && warp == 0) {
    double at = 0.0, au = 0.0;
    for (int u = lane; u < npp; u += 32) {
      at += (double)s_xv[u] * (double)s_del[u];
      au += (double)s_xv[u] * (double)s_delu[u];
    }
    for (int o = 16; o; o >>= 1) {
      at += __shfl_down_sync(0xffffffffu, at, o);
      au += __shfl_down_sync(0xffffffffu, au, o);
    }
    if (lane == 0) {
      xpart[((int64_t)b * 2) * nchunks] += at;
      xpart[((int64_t)b * 2 + 1) * nchunks] += au;
    }
  }
  if (!fix_dots) return;
  const float* Vb = V + (int64_t)b * M * ld;
  for (int j = warp; j < m; j += APPLY_THREADS / 32) {
    double acc = 0.0, accu = 0.0;
    for (int u = lane; u < npp; u += 32) {
      const double v = (double)Vb[(int64_t)j * ld + s_i[u]];
      acc += v * (double)s_del[u];
      if (olsen) accu += v * (double)s_delu[u];
    }
    for (int o = 16; o; o >>= 1) {
      acc += __shfl_down_sync(0xffffffffu, acc, o);
      accu += __shfl_down_sync(0xffffffffu, accu, o);
    }
    if (lane == 0) {
      partial[((int64_t)b * m + j) * nchunks] += acc;
      if (olsen) upart[((int64_t)b * m + j) * nchunks] += accu;
    }
  }
}

}  // namespace

int pspace_size(const BinProblem& bp, int requested) {
  if (requested <= 0) return 0;
  const int64_t ncan = (int64_t)bp.nstr * (bp.nstr + 1) / 2;
  const int64_t cap = std::min<int64_t>({(int64_t)requested, (int64_t)PSP_MAX, ncan / 2});
  if (cap < 2) return 0;
  if (eig_layout(bp.n).total + 4096 > 227u * 1024u) return 0;
  return (int)cap;
}

void pspace_setup(mbe_ctx* ctx, BinProblem& bp, const float* hd, int64_t ld, double shift,
                  int npp, PspaceWork& w) {
  w.npp = npp;
  if (!npp) return;
  const int B = bp.B;
  w.sel.reset(&ctx->pool, (size_t)B * PSP_MAX);
  w.lam.reset(&ctx->pool, (size_t)B * PSP_MAX);
  w.U.reset(&ctx->pool, (size_t)B * PSP_MAX * PSP_MAX);
  cudaStream_t st = ctx->stream;
  k_psp_select<<<B, SEL_THREADS, 0, st>>>(hd, bp.nstr, ld, npp, w.sel.ptr);
  CU_LAUNCH_CHECK();
  const uint32_t smem = eig_layout(bp.n).total;
  static bool attr_set[MBE_MAX_DEVICES] = {false};
  once_per_device(attr_set, ctx->device, [] {
    CU_CHECK(cudaFuncSetAttribute(k_psp_eigh, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  227 * 1024 - 4096));
    CU_CHECK(cudaFuncSetAttribute(k_psp_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  PSP_MAX * PSP_PITCH * 4));
  });
  k_psp_eigh<<<B, EIG_THREADS, smem, st>>>(bp.tab->masks.ptr, bp.nstr, bp.n, bp.nsig,
                                           bp.heff.ptr, bp.hp.ptr, bp.gp.ptr, hd, ld,
                                           (float)shift, npp, w.sel.ptr, w.lam.ptr, w.U.ptr);
  CU_LAUNCH_CHECK();
}

void pspace_apply(mbe_ctx* ctx, const BinProblem& bp, const PspaceWork& w, float* T,
                  const float* hd, int64_t ld, const double* theta, const float* V, int m, int M,
                  int nchunks, double* partial, bool fix_dots, const int32_t* active,
                  bool olsen, float* Uo, const float* X, double* upart, double* xpart) {
  if (!w.npp) return;
  const uint32_t smem = (uint32_t)w.npp * PSP_PITCH * 4;
  k_psp_apply<<<bp.B, APPLY_THREADS, smem, ctx->stream>>>(
      T, hd, bp.nstr, ld, theta, w.npp, w.sel.ptr, w.U.ptr, w.lam.ptr, V, m, M, nchunks, partial,
      fix_dots ? 1 : 0, active, olsen ? 1 : 0, Uo, X, upart, xpart);
  CU_LAUNCH_CHECK();
}
